"""GB300-native EFIE/RWG impedance-matrix fill with the adaptive Green / Exp
interpolation tables of Yang & Su, "Fast Green Function Evaluation for Method
of Moment". The work is done by libgfmom (C-ABI, include/gfmom.h); this
package only binds it. Importing does not load the library; the first call
does (and fails loudly if it cannot).
"""
from .gfmom import (GF_EXP, GF_FP32, GF_FP64, GF_GREEN, GF_OP_EFIE, GF_OP_MFIE, GF_PART_MIRROR, GF_PART_NEAR,
                    GF_PART_PAIRS, GF_PART_REGULAR, GF_PART_ZERO, Sparse, gf_fill_mfie,
                    Batch, GfError, Mesh, Table, fill, gf_batch_config, gf_batch_create, gf_batch_destroy,
                    gf_batch_launch, efie_fill, gf_excitation, gf_far_field, gf_fill, gf_fill_backward,
                    gf_fill_parts, planewave_rcs,
                    gf_last_error, gf_mesh_create, gf_mesh_destroy, gf_mesh_edges, gf_mesh_info,
                    gf_mesh_set_vertices, gf_params, gf_params_default, gf_range, gf_table_create,
                    gf_table_destroy, gf_table_eval, gf_table_info, gf_table_nodes, lib, gf_table_eval_host,
                    gf_table_create_for_mesh, gf_fill_batched)

__all__ = ["GF_EXP", "GF_FP32", "GF_FP64", "GF_GREEN", "GF_OP_EFIE", "GF_OP_MFIE", "GF_PART_MIRROR", "GF_PART_NEAR",
           "GF_PART_PAIRS", "GF_PART_REGULAR",
           "GF_PART_ZERO", "Sparse", "gf_fill_mfie",
           "Batch", "GfError", "Mesh", "Table", "fill", "gf_batch_config", "gf_batch_create", "gf_batch_destroy",
           "gf_batch_launch", "efie_fill", "gf_excitation", "gf_far_field", "gf_fill", "gf_fill_backward",
           "gf_fill_parts", "planewave_rcs",
           "gf_last_error", "gf_mesh_create", "gf_mesh_destroy", "gf_mesh_edges", "gf_mesh_info",
           "gf_mesh_set_vertices", "gf_params", "gf_params_default", "gf_range", "gf_table_create",
           "gf_table_destroy", "gf_table_eval", "gf_table_info", "gf_table_nodes", "lib", "gf_table_eval_host",
           "gf_table_create_for_mesh", "gf_fill_batched"]
