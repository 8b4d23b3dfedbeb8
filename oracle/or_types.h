// Scalar, complex and 3-vector types of the oracle. The fill is written once
// for a scalar type T: double for values, Dual<N> for forward-mode gradients.
// Test infrastructure only (see oracle.h).
#ifndef GF_OR_TYPES_H
#define GF_OR_TYPES_H
#include <cmath>

namespace orc {

// ---- forward-mode dual number with N directional derivatives --------------
template <int N>
struct Dual {
  double v;
  double d[N];
  Dual() : v(0) { for (int i = 0; i < N; ++i) d[i] = 0; }
  Dual(double x) : v(x) { for (int i = 0; i < N; ++i) d[i] = 0; }
  static Dual var(double x, int dir) { Dual r(x); r.d[dir] = 1.0; return r; }
};
template <int N> inline Dual<N> operator+(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r(a.v + b.v); for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i]; return r; }
template <int N> inline Dual<N> operator-(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r(a.v - b.v); for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i]; return r; }
template <int N> inline Dual<N> operator-(const Dual<N>& a) {
  Dual<N> r(-a.v); for (int i = 0; i < N; ++i) r.d[i] = -a.d[i]; return r; }
template <int N> inline Dual<N> operator*(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r(a.v * b.v); for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i]; return r; }
template <int N> inline Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r(a.v / b.v);
  for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / (b.v * b.v);
  return r; }
template <int N> inline Dual<N> operator+(const Dual<N>& a, double b) { return a + Dual<N>(b); }
template <int N> inline Dual<N> operator+(double a, const Dual<N>& b) { return Dual<N>(a) + b; }
template <int N> inline Dual<N> operator-(const Dual<N>& a, double b) { return a - Dual<N>(b); }
template <int N> inline Dual<N> operator-(double a, const Dual<N>& b) { return Dual<N>(a) - b; }
template <int N> inline Dual<N> operator*(const Dual<N>& a, double b) {
  Dual<N> r(a.v * b); for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b; return r; }
template <int N> inline Dual<N> operator*(double a, const Dual<N>& b) { return b * a; }
template <int N> inline Dual<N> operator/(const Dual<N>& a, double b) { return a * (1.0 / b); }
template <int N> inline Dual<N> operator/(double a, const Dual<N>& b) { return Dual<N>(a) / b; }
template <int N> inline Dual<N> sqrt(const Dual<N>& a) {
  double s = std::sqrt(a.v); Dual<N> r(s);
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] / (2.0 * s); return r; }
template <int N> inline Dual<N> sin(const Dual<N>& a) {
  Dual<N> r(std::sin(a.v)); double c = std::cos(a.v);
  for (int i = 0; i < N; ++i) r.d[i] = c * a.d[i]; return r; }
template <int N> inline Dual<N> cos(const Dual<N>& a) {
  Dual<N> r(std::cos(a.v)); double s = -std::sin(a.v);
  for (int i = 0; i < N; ++i) r.d[i] = s * a.d[i]; return r; }
template <int N> inline Dual<N> atan2(const Dual<N>& y, const Dual<N>& x) {
  Dual<N> r(std::atan2(y.v, x.v)); double q = x.v * x.v + y.v * y.v;
  for (int i = 0; i < N; ++i) r.d[i] = (x.v * y.d[i] - y.v * x.d[i]) / q; return r; }
template <int N> inline Dual<N> log(const Dual<N>& a) {
  Dual<N> r(std::log(a.v));
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] / a.v; return r; }
template <int N> inline Dual<N> asinh(const Dual<N>& a) {
  Dual<N> r(std::asinh(a.v)); double q = 1.0 / std::sqrt(1.0 + a.v * a.v);
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * q; return r; }
template <int N> inline Dual<N> cosh(const Dual<N>& a) {
  Dual<N> r(std::cosh(a.v)); double q = std::sinh(a.v);
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * q; return r; }
template <int N> inline Dual<N> fabs(const Dual<N>& a) { return a.v < 0 ? -a : a; }
template <int N> inline double val(const Dual<N>& a) { return a.v; }
inline double val(double a) { return a; }

// ---- complex over T ---------------------------------------------------------
template <class T>
struct Cx {
  T re, im;
  Cx() : re(0.0), im(0.0) {}
  explicit Cx(double r) : re(r), im(0.0) {}
  Cx(T r, T i) : re(r), im(i) {}
};
template <class T> inline Cx<T> operator+(const Cx<T>& a, const Cx<T>& b) { return Cx<T>(a.re + b.re, a.im + b.im); }
template <class T> inline Cx<T> operator-(const Cx<T>& a, const Cx<T>& b) { return Cx<T>(a.re - b.re, a.im - b.im); }
template <class T> inline Cx<T> operator*(const Cx<T>& a, const Cx<T>& b) {
  return Cx<T>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re); }
template <class T> inline Cx<T> operator*(const Cx<T>& a, const T& s) { return Cx<T>(a.re * s, a.im * s); }
template <class T> inline Cx<T> operator*(const T& s, const Cx<T>& a) { return Cx<T>(a.re * s, a.im * s); }
template <class T> inline Cx<T>& operator+=(Cx<T>& a, const Cx<T>& b) { a.re = a.re + b.re; a.im = a.im + b.im; return a; }

// ---- 3-vector over T --------------------------------------------------------
template <class T>
struct V3 {
  T x, y, z;
  V3() : x(), y(), z() {}
  V3(T a, T b, T c) : x(a), y(b), z(c) {}
};
template <class T> inline V3<T> operator+(const V3<T>& a, const V3<T>& b) { return V3<T>(a.x + b.x, a.y + b.y, a.z + b.z); }
template <class T> inline V3<T> operator-(const V3<T>& a, const V3<T>& b) { return V3<T>(a.x - b.x, a.y - b.y, a.z - b.z); }
template <class T> inline V3<T> operator*(const V3<T>& a, const T& s) { return V3<T>(a.x * s, a.y * s, a.z * s); }
template <class T> inline V3<T> operator*(const T& s, const V3<T>& a) { return a * s; }
template <class T> inline T dot(const V3<T>& a, const V3<T>& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class T> inline V3<T> cross(const V3<T>& a, const V3<T>& b) {
  return V3<T>(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x); }
template <class T> inline T norm(const V3<T>& a) { using std::sqrt; return sqrt(dot(a, a)); }

}  // namespace orc
#endif
