// Device-side layouts and per-element bodies of the sm_103a library.
//
// Every kernel of the library is a thin __global__ wrapper that maps a thread
// to one element (cell, face or cross-section cell) of a box and calls one of
// the bodies below.  All arithmetic is FP64.  Equation and section numbers
// refer to arXiv 2303.10785.
#pragma once
#include <cmath>
#include <cstdint>
#include <cstring>
#include <type_traits>

#ifdef __CUDACC__
#define GBR_HD __host__ __device__ __forceinline__
#else
#define GBR_HD inline
#endif

namespace gbr {

constexpr int H = 6;   // halo of primitive-derived arrays: an interface needs cells i-5..i+6
constexpr int E = 10;  // geometry extension: metric derivative (reach 5) of products that are themselves
                       // metric derivatives (reach 5)

// ---------------------------------------------------------------------------
// Layouts
// ---------------------------------------------------------------------------
struct Layout {
  int nd, nv;
  int n[3];
  int per[3];
  int hp[3];          // halo per axis (H on active axes)
  int pn[3];          // padded extents
  long long ps[3];    // padded strides
  long long pcount;
  int he[3];          // geometry extension per axis (E on active axes; kExtIG4 on periodic axes of a
                      // MIG4 grid, whose metric operators solve IG4 over the unwrapped line)
  int cg[3];          // cell metrics kept on [-cg, n + cg) (5; kExtIG4 - 10 with the long lines; 0 closed)
  int en[3];
  long long es[3];
  long long ecount;
  int fn[3][3];       // face-array extents for direction d
  long long fs[3][3]; // face-array strides
  long long fcount[3];
  long long ncells;
  int nn[3];          // extended node extents (n + 2E + 1 on active axes, n + 1 on closed ones)
  long long ns[3];
  long long ncount;
  int closed[3];      // wall-bounded axis without ghost nodes: no geometry extension, App. C operators
};

// MIG4 geometry: extension of a periodic axis (IG4 on the unbounded unwrapped line: the inverse of the
// (alpha, 1, alpha) operator decays by 0.4226 per cell, so the end rows of a line this long reach the
// cells that are kept below 1e-20 of their own size)
constexpr int kExtIG4 = 64;

// ig4_geo: per axis, 1 when the metrics are built with IG4 on the long unwrapped line
inline Layout make_layout(int nd, const int* n, const int* periodic, const int* closed, const int* ig4_geo) {
  Layout L;
  L.nd = nd;
  L.nv = nd + 2;
  for (int d = 0; d < 3; ++d) {
    bool act = d < nd;
    L.n[d] = act ? n[d] : 1;
    L.per[d] = act ? periodic[d] : 1;
    L.closed[d] = act && !periodic[d] && closed[d];
    L.hp[d] = act ? H : 0;
    L.pn[d] = L.n[d] + 2 * L.hp[d];
    L.he[d] = (act && !L.closed[d]) ? ((periodic[d] && ig4_geo[d]) ? kExtIG4 : E) : 0;
    L.cg[d] = !act ? 0 : (L.closed[d] ? 0 : ((periodic[d] && ig4_geo[d]) ? kExtIG4 - 10 : 5));
    L.en[d] = L.n[d] + 2 * L.he[d];
    L.nn[d] = act ? L.n[d] + 2 * L.he[d] + 1 : 1;
  }
  L.ps[0] = 1;
  L.ps[1] = L.pn[0];
  L.ps[2] = (long long)L.pn[0] * L.pn[1];
  L.pcount = L.ps[2] * L.pn[2];
  L.es[0] = 1;
  L.es[1] = L.en[0];
  L.es[2] = (long long)L.en[0] * L.en[1];
  L.ecount = L.es[2] * L.en[2];
  L.ns[0] = 1;
  L.ns[1] = L.nn[0];
  L.ns[2] = (long long)L.nn[0] * L.nn[1];
  L.ncount = L.ns[2] * L.nn[2];
  L.ncells = (long long)L.n[0] * L.n[1] * L.n[2];
  for (int d = 0; d < 3; ++d) {
    for (int e = 0; e < 3; ++e) L.fn[d][e] = L.n[e] + ((e == d && d < nd) ? 1 : 0);
    L.fs[d][0] = 1;
    L.fs[d][1] = L.fn[d][0];
    L.fs[d][2] = (long long)L.fn[d][0] * L.fn[d][1];
    L.fcount[d] = L.fs[d][2] * L.fn[d][2];
  }
  return L;
}

GBR_HD long long pidx(const Layout& L, int i, int j, int k) {
  return (long long)(i + L.hp[0]) + (long long)(j + L.hp[1]) * L.ps[1] + (long long)(k + L.hp[2]) * L.ps[2];
}
GBR_HD long long eidx(const Layout& L, int i, int j, int k) {
  return (long long)(i + L.he[0]) + (long long)(j + L.he[1]) * L.es[1] + (long long)(k + L.he[2]) * L.es[2];
}
GBR_HD long long nidx(const Layout& L, int i, int j, int k) {
  return (long long)(i + L.he[0]) + (long long)(j + L.he[1]) * L.ns[1] + (long long)(k + L.he[2]) * L.ns[2];
}
GBR_HD long long cidx(const Layout& L, int i, int j, int k) {
  return (long long)i + (long long)j * L.n[0] + (long long)k * L.n[0] * L.n[1];
}
// interface i+1/2 along d (i in [-1, n_d - 1]) of the cross-section cell (j, k)
GBR_HD long long fidx(const Layout& L, int d, int i, int j, int k) {
  int c[3] = {i, j, k};
  c[d] += 1;
  return (long long)c[0] + (long long)c[1] * L.fs[d][1] + (long long)c[2] * L.fs[d][2];
}
// The same indices in 32-bit unsigned arithmetic, for the interface kernels: every offset into
// one of their arrays (field x padded cell, component x interface) is below 2^32, which
// valid_params checks for every context (a grid with more cells would not fit in device
// memory).  One widening multiply-add per address instead of 64-bit index arithmetic.
GBR_HD unsigned pidx32(const Layout& L, int i, int j, int k) {
  return (unsigned)(i + L.hp[0]) + (unsigned)(j + L.hp[1]) * (unsigned)L.ps[1] +
         (unsigned)(k + L.hp[2]) * (unsigned)L.ps[2];
}
GBR_HD unsigned fidx32(const Layout& L, int d, int i, int j, int k) {
  int c[3] = {i, j, k};
  c[d] += 1;
  return (unsigned)c[0] + (unsigned)c[1] * (unsigned)L.fs[d][1] + (unsigned)c[2] * (unsigned)L.fs[d][2];
}
// Index type of the interface kernels: 32-bit offsets in FP64 (1.4 % faster: the FP64 kernel issues
// its integer work beside a busy FP64 pipe), 64-bit in FP32 (32-bit offsets measured 40 % slower
// there).
template <class R>
using FaceIx = std::conditional_t<sizeof(R) == sizeof(double), unsigned, long long>;
template <class I>
GBR_HD I face_pidx(const Layout& L, int i, int j, int k) {
  if constexpr (sizeof(I) == 4) return pidx32(L, i, j, k);
  else return pidx(L, i, j, k);
}
template <class I>
GBR_HD I face_fidx(const Layout& L, int d, int i, int j, int k) {
  if constexpr (sizeof(I) == 4) return fidx32(L, d, i, j, k);
  else return fidx(L, d, i, j, k);
}

struct Box {
  int lo[3], hi[3];
};
GBR_HD long long box_size(const Box& b) {
  return (long long)(b.hi[0] - b.lo[0]) * (b.hi[1] - b.lo[1]) * (b.hi[2] - b.lo[2]);
}
// (i, j, k) of the t-th cell of a box, i fastest.  (The 64-bit divisions stay: the same decode in
// 32-bit arithmetic made the FP32 interface kernel 51 % slower -- 3.3x the long-scoreboard stalls
// in ncu -- and changed nothing elsewhere.)
GBR_HD void box_coord(const Box& b, long long t, int& i, int& j, int& k) {
  const long long nx = b.hi[0] - b.lo[0], ny = b.hi[1] - b.lo[1];
  i = b.lo[0] + (int)(t % nx);
  t /= nx;
  j = b.lo[1] + (int)(t % ny);
  k = b.lo[2] + (int)(t / ny);
}

struct Phys {
  double gamma, gm1, igm1;
  double mu_ref, suth_s, it_ref;
  double alpha_d;            // alpha^D
  double mp_alpha, mp_beta, mp_eps;
  double kfac;               // kappa = mu * kfac, kfac = gamma / ((gamma - 1) Pr)
  double dt_visc_fac;        // max(4/3, gamma/Pr) of the viscous time-step bound
  int viscous, sutherland;
};

// ---------------------------------------------------------------------------
// Math helpers
// ---------------------------------------------------------------------------
GBR_HD double grsqrt(double x) {
#ifdef __CUDA_ARCH__
  return rsqrt(x);
#else
  return 1.0 / std::sqrt(x);
#endif
}
// 1/x by Newton's method for the reciprocal, y <- y + y (1 - x y), from the hardware's approximate
// reciprocal (PTX rcp.approx.ftz.f64, relative error below 2^-22): the error squares at each step,
// so two steps leave it below the FP64 rounding (within one unit in the last place of 1/x; the
// FP64 division is correctly rounded).  Four FMAs against the division's longer sequence on the
// FP64 pipe.  For finite, nonzero, normal x (densities, a Riemann fan's width, S - S*); gbr_check_rcp
// measures it against the division.
GBR_HD double grcp(double x) {
#ifdef __CUDA_ARCH__
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  double e = fma(-x, y, 1.0);
  y = fma(y, e, y);
  e = fma(-x, y, 1.0);
  return fma(y, e, y);
#else
  return 1.0 / x;
#endif
}
// FP32 (mixed path): the division (its FP32 sequence is short)
GBR_HD float grcp(float x) { return 1.0f / x; }
// a / b: FP64 as a times grcp(b), FP32 the division
GBR_HD double gdiv(double a, double b) { return a * grcp(b); }
GBR_HD float gdiv(float a, float b) { return a / b; }

GBR_HD double gfma(double a, double b, double c) {
#ifdef __CUDA_ARCH__
  return fma(a, b, c);
#else
  return a * b + c;
#endif
}
// Comparisons, min/max, |x| and minmod on the bit patterns of doubles.  On a
// B300 the FP64 pipe issues 2 instructions/clk/SM while the integer pipe issues
// 64, so the limiter's and the Riemann solver's branch logic is kept off the
// FP64 pipe.  The key below is monotone in the value and maps +0 and -0 to the
// same key, so key(a) < key(b) is exactly a < b for every non-NaN pair.  On the
// device the double -> bits move is an opaque register move: a plain
// reinterpret lets the compiler fold "bits & mask" or a select of reinterpreted
// values back into FP64 |x| / negate / select instructions, which run on the
// FP64 pipe again.
GBR_HD long long dbits(double x) {
#ifdef __CUDA_ARCH__
  long long r;
  asm("mov.b64 %0, %1;" : "=l"(r) : "d"(x));
  return r;
#else
  long long r;
  std::memcpy(&r, &x, sizeof r);
  return r;
#endif
}
GBR_HD double bitsd(long long b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double(b);
#else
  double r;
  std::memcpy(&r, &b, sizeof r);
  return r;
#endif
}
constexpr long long kMag = 0x7fffffffffffffffLL;
constexpr long long kSign = (long long)0x8000000000000000ULL;
// order key of a bit pattern
GBR_HD long long bkey(long long b) { return b < 0 ? -(b & kMag) : b; }
GBR_HD long long okey(double x) { return bkey(dbits(x)); }
// min / max of two bit patterns by value, exactly like a < b ? a : b and
// a > b ? a : b on the doubles (a tie returns the second argument)
GBR_HD long long bmin(long long a, long long b) { return bkey(a) < bkey(b) ? a : b; }
GBR_HD long long bmax(long long a, long long b) { return bkey(b) < bkey(a) ? a : b; }
// App. E: minmod(a, b) = 1/2 (sign a + sign b) min(|a|, |b|), i.e. the smaller-magnitude
// argument when both have the same sign, else a zero; when one argument is zero
// the product with the sign sum keeps that sum's sign (-0 for a negative sum).
GBR_HD long long bminmod(long long a, long long b) {
  const long long ma = a & kMag, mb = b & kMag;
  const long long m = ma < mb ? ma : mb;  // |a| < |b| ? |a| : |b|
  const int sa = a > 0 ? 1 : ((a < 0 && ma != 0) ? -1 : 0);
  const int sb = b > 0 ? 1 : ((b < 0 && mb != 0) ? -1 : 0);
  const int sum = sa + sb;
  return sum == 2 ? m : (sum == -2 ? (m | kSign) : (sum < 0 ? kSign : 0LL));
}
GBR_HD bool dlt(double a, double b) { return okey(a) < okey(b); }
GBR_HD bool dle(double a, double b) { return okey(a) <= okey(b); }
GBR_HD bool is_pos(double x) { return dbits(x) > 0; }                       // x > 0
GBR_HD bool is_neg(double x) { return (dbits(x) & kMag) != 0 && dbits(x) < 0; }  // x < 0
GBR_HD double gmin(double a, double b) { return bitsd(bmin(dbits(a), dbits(b))); }  // a < b ? a : b
GBR_HD double gmax(double a, double b) { return bitsd(bmax(dbits(a), dbits(b))); }  // a > b ? a : b
GBR_HD double gabs(double x) { return bitsd(dbits(x) & kMag); }
GBR_HD double minmod(double a, double b) { return bitsd(bminmod(dbits(a), dbits(b))); }

// Composite stencils of the MEG6 interface operators (Sec. 7): the interface
// value I(f)_{i+1/2} = avg of the van Leer left/right states built from E6
// gradients and the gradient-based second derivative, and the derivative
// D(f)_i = I(f)_{i+1/2} - I(f)_{i-1/2}.  The D weights 2282, -546, 89, -3, -1
// (over 2880) are the ones printed in the Sec. 7 proof; the I weights follow
// from the same three formulas: 1821, -461, 85, -4, -1 (over 2880) on
// (f_i + f_{i+1}), (f_{i-1} + f_{i+2}), ... .
constexpr double kD1 = 2282.0 / 2880.0, kD2 = -546.0 / 2880.0, kD3 = 89.0 / 2880.0, kD4 = -3.0 / 2880.0,
                 kD5 = -1.0 / 2880.0;
constexpr double kI0 = 1821.0 / 2880.0, kI1 = -461.0 / 2880.0, kI2 = 85.0 / 2880.0, kI3 = -4.0 / 2880.0,
                 kI4 = -1.0 / 2880.0;

GBR_HD double stencil_D(const double* f, long long e, long long s) {
  double r = kD1 * (f[e + s] - f[e - s]);
  r = gfma(kD2, f[e + 2 * s] - f[e - 2 * s], r);
  r = gfma(kD3, f[e + 3 * s] - f[e - 3 * s], r);
  r = gfma(kD4, f[e + 4 * s] - f[e - 4 * s], r);
  r = gfma(kD5, f[e + 5 * s] - f[e - 5 * s], r);
  return r;
}
// interface between e and e + s
GBR_HD double stencil_I(const double* f, long long e, long long s) {
  double r = kI0 * (f[e] + f[e + s]);
  r = gfma(kI1, f[e - s] + f[e + 2 * s], r);
  r = gfma(kI2, f[e - 2 * s] + f[e + 3 * s], r);
  r = gfma(kI3, f[e - 3 * s] + f[e + 4 * s], r);
  r = gfma(kI4, f[e - 4 * s] + f[e + 5 * s], r);
  return r;
}
// product stencil: D applied to the pointwise product a * b
GBR_HD double stencil_D_prod(const double* a, const double* b, long long e, long long s) {
  const double c[5] = {kD1, kD2, kD3, kD4, kD5};
  double r = 0.0;
  for (int m = 1; m <= 5; ++m) r = gfma(c[m - 1], a[e + m * s] * b[e + m * s] - a[e - m * s] * b[e - m * s], r);
  return r;
}

// ---------------------------------------------------------------------------
// App. C on a wall-bounded (closed) axis of n cells, used for every cell of such an axis:
// f' second-order one-sided at the end cells, fourth-order biased next to them (the printed stencil shifted back by one index),
// fourth-order central third, E6 inside; f'' one-sided from f' at the two end cells, the
// interior formula elsewhere; interface values: the wall interfaces take the boundary cell's
// own state, the interfaces between the first (last) two cells the inner cell's state, the
// others the mean of both van Leer states.  `f(m)` reads cell m of the line.
// ---------------------------------------------------------------------------
template <class F>
GBR_HD double appc_d1(const F& f, int m, int n) {
  if (m == 0) return -1.5 * f(0) + 2.0 * f(1) - 0.5 * f(2);
  if (m == n - 1) return 1.5 * f(n - 1) - 2.0 * f(n - 2) + 0.5 * f(n - 3);
  if (m == 1) return -0.25 * f(0) - (5.0 / 6.0) * f(1) + 1.5 * f(2) - 0.5 * f(3) + f(4) * (1.0 / 12.0);
  if (m == n - 2)
    return 0.25 * f(n - 1) + (5.0 / 6.0) * f(n - 2) - 1.5 * f(n - 3) + 0.5 * f(n - 4) - f(n - 5) * (1.0 / 12.0);
  if (m == 2 || m == n - 3) return (2.0 / 3.0) * (f(m + 1) - f(m - 1)) - (f(m + 2) - f(m - 2)) * (1.0 / 12.0);
  double r = (3.0 / 4.0) * (f(m + 1) - f(m - 1));
  r = gfma(-3.0 / 20.0, f(m + 2) - f(m - 2), r);
  return gfma(1.0 / 60.0, f(m + 3) - f(m - 3), r);
}
template <class F>
GBR_HD double appc_d2(const F& f, int m, int n) {
  auto d1 = [&](int c) { return appc_d1(f, c, n); };
  if (m == 0) return -1.5 * d1(0) + 2.0 * d1(1) - 0.5 * d1(2);
  if (m == n - 1) return 1.5 * d1(n - 1) - 2.0 * d1(n - 2) + 0.5 * d1(n - 3);
  if (m == 1) return -0.25 * d1(0) - (5.0 / 6.0) * d1(1) + 1.5 * d1(2) - 0.5 * d1(3) + d1(4) * (1.0 / 12.0);
  if (m == n - 2)
    return 0.25 * d1(n - 1) + (5.0 / 6.0) * d1(n - 2) - 1.5 * d1(n - 3) + 0.5 * d1(n - 4) - d1(n - 5) * (1.0 / 12.0);
  return 2.0 * (f(m + 1) - 2.0 * f(m) + f(m - 1)) - 0.5 * (d1(m + 1) - d1(m - 1));
}
// interface m + 1/2, m in [-1, n - 1]
template <class F>
GBR_HD double appc_face(const F& f, int m, int n) {
  auto plus = [&](int c) { return f(c) + 0.5 * appc_d1(f, c, n) + appc_d2(f, c, n) * (1.0 / 12.0); };
  auto minus = [&](int c) { return f(c) - 0.5 * appc_d1(f, c, n) + appc_d2(f, c, n) * (1.0 / 12.0); };
  if (m == -1 || m == 0) return minus(m + 1);
  if (m == n - 1 || m == n - 2) return plus(m);
  return 0.5 * (plus(m) + minus(m + 1));
}
template <class F>
GBR_HD double appc_D(const F& f, int m, int n) { return appc_face(f, m, n) - appc_face(f, m - 1, n); }

// cell index of (i, j, k) along d and the extended index of cell 0 of that line
GBR_HD int line_pos(int d, int i, int j, int k) { return d == 0 ? i : (d == 1 ? j : k); }
GBR_HD long long line_base(const Layout& L, int d, int i, int j, int k) {
  int c[3] = {i, j, k};
  c[d] = 0;
  return eidx(L, c[0], c[1], c[2]);
}

// ---------------------------------------------------------------------------
// MIG4 metric operators (Sec. 7 step 2: the metric derivative and interpolation use the scheme's
// own gradients; for MIG4 x' is the IG4 system of Eq. IG4_grads).  A geometry line is solved as a
// whole with the explicit end rows (second-order one-sided, fourth-order biased, fourth-order
// central at the three end points of each side, IG4 rows between); on periodic axes the line is
// the unwrapped line extended kExtIG4 cells beyond each side, i.e. IG4 on the unbounded line.
// ---------------------------------------------------------------------------
// Eq. IG4_grads: alpha = 5/14
constexpr double kIg4Alpha = 5.0 / 14.0;

// one line of an extended-box array: cell x of the line at p[x * s] (x may be negative)
struct LineRef {
  double* p;
  long long s;
  GBR_HD double& operator()(int x) const { return p[x * s]; }
};

// Thomas factors of the open-line system of m rows, the same for every line of that length:
// t[r] = c'_r, t[m + r] = the pivot b_r - a_r c'_{r-1}
GBR_HD void ig4_geo_factor(double* t, int m) {
  double cp = 0.0;
  for (int r = 0; r < m; ++r) {
    const bool expl = r < 3 || r >= m - 3;
    const double a = expl ? 0.0 : kIg4Alpha, c = expl ? 0.0 : kIg4Alpha;
    const double den = 1.0 - (r > 0 ? a * cp : 0.0);
    cp = c / den;
    t[r] = cp;
    t[m + r] = den;
  }
}

// IG4 derivative w(x) of the line values f(x), x in [lo, hi), with the explicit end rows
template <class F>
GBR_HD void ig4_geo_solve(const F& f, const LineRef& w, int lo, int hi, const double* t) {
  const int m = hi - lo, e = hi - 1;
  const double al = kIg4Alpha;
  const double c1 = (2.0 + al) / 3.0, c2 = (4.0 * al - 1.0) / 12.0;
  double rp = 0.0;
  for (int r = 0; r < m; ++r) {
    const int x = lo + r;
    double rhs;
    if (r == 0) rhs = -1.5 * f(x) + 2.0 * f(x + 1) - 0.5 * f(x + 2);
    else if (r == 1) rhs = -0.25 * f(x - 1) - (5.0 / 6.0) * f(x) + 1.5 * f(x + 1) - 0.5 * f(x + 2) + f(x + 3) / 12.0;
    else if (r == 2) rhs = (2.0 / 3.0) * (f(x + 1) - f(x - 1)) - (f(x + 2) - f(x - 2)) / 12.0;
    else if (x == e) rhs = 1.5 * f(e) - 2.0 * f(e - 1) + 0.5 * f(e - 2);
    else if (x == e - 1)
      rhs = 0.25 * f(e) + (5.0 / 6.0) * f(e - 1) - 1.5 * f(e - 2) + 0.5 * f(e - 3) - f(e - 4) / 12.0;
    else if (x == e - 2) rhs = (2.0 / 3.0) * (f(e - 1) - f(e - 3)) - (f(e) - f(e - 4)) / 12.0;
    else rhs = c1 * (f(x + 1) - f(x - 1)) + c2 * (f(x + 2) - f(x - 2));
    const double a = (r < 3 || r >= m - 3) ? 0.0 : al;
    rp = (rhs - a * rp) / t[m + r];
    w(x) = rp;
  }
  double xn = 0.0;
  for (int r = m - 1; r >= 0; --r) {
    const int x = lo + r;
    xn = (r == m - 1) ? w(x) : w(x) - t[r] * xn;
    w(x) = xn;
  }
}

// interface value at x + 1/2 (Eq. FP-interp, interp-formulae): the mean of the van Leer states of
// cells x and x + 1 from f, its IG4 derivative w and f'' = 2 (f_{x+1} - 2 f_x + f_{x-1}) - (w_{x+1} - w_{x-1}) / 2
template <class F>
GBR_HD double ig4_geo_face(const F& f, const LineRef& w, int x) {
  auto f2 = [&](int y) { return 2.0 * (f(y + 1) - 2.0 * f(y) + f(y - 1)) - 0.5 * (w(y + 1) - w(y - 1)); };
  const double left = f(x) + 0.5 * w(x) + f2(x) / 12.0;
  const double right = f(x + 1) - 0.5 * w(x + 1) + f2(x + 1) / 12.0;
  return 0.5 * (left + right);
}

// ---------------------------------------------------------------------------
// Geometry bodies (Sec. 3, Sec. 4, Sec. 7)
// ---------------------------------------------------------------------------
struct GeoArgs {
  Layout L;
  const double* nodes;  // [nd][ncount]  extended nodes
  const double* nvel;   // [nd][ncount]  extended node velocities (moving) or null
  double* xc;           // [nd][ecount]  centroids
  double* vc;           // [nd][ecount]  centroid velocities
  double* xd;           // [9][ecount]   xd[a*3+d] = D_d x_a
  double* mh;           // [9][ecount]   hat metrics mh[e*3+a]
  double* det;          // [ecount]      1/J
  double* mu;           // [9][ecount]   unhatted metrics (viscous)
  double* mt;           // [3][ecount]   hat time metrics (moving)
  double* fh[3];        // [nd][fcount]
  double* fu[3];        // [nd*nd][fcount]
  double* ft[3];        // [fcount]
  double* gcl;          // [ncells]
  double* jac;          // [ncells]  J = 1/(1/J)
  int viscous, moving;
};

// Sec. 3: cell centroid = average of the cell's vertices
GBR_HD void body_centroid(const GeoArgs& G, int i, int j, int k) {
  const Layout& L = G.L;
  const int nd = L.nd;
  const long long e = eidx(L, i, j, k);
  const double inv = (nd == 3) ? 0.125 : 0.25;
  for (int a = 0; a < nd; ++a) {
    const double* X = G.nodes + a * L.ncount;
    double s = 0.0, sv = 0.0;
    for (int ck = 0; ck < (nd == 3 ? 2 : 1); ++ck)
      for (int cj = 0; cj < 2; ++cj)
        for (int ci = 0; ci < 2; ++ci) {
          const long long m = nidx(L, i + ci, j + cj, k + ck);
          s = s + X[m];
          if (G.moving) sv = sv + G.nvel[a * L.ncount + m];
        }
    G.xc[a * L.ecount + e] = s * inv;
    if (G.moving) G.vc[a * L.ecount + e] = sv * inv;
  }
}

// Sec. 7 step 2: consistent derivative of the coordinates, xd[a][d] = D_d(x_a)
GBR_HD void body_coord_derivative(const GeoArgs& G, int d, int i, int j, int k) {
  const Layout& L = G.L;
  const long long e = eidx(L, i, j, k);
  for (int a = 0; a < L.nd; ++a) {
    const double* x = G.xc + a * L.ecount;
    double v;
    if (L.closed[d]) {
      const long long b = line_base(L, d, i, j, k), s = L.es[d];
      v = appc_D([&](int m) { return x[b + m * s]; }, line_pos(d, i, j, k), L.n[d]);
    } else {
      v = stencil_D(x, e, L.es[d]);
    }
    G.xd[(a * 3 + d) * L.ecount + e] = v;
  }
}

// D along d of the product a * b (Sec. 7 step 2), App. C on a closed axis
GBR_HD double metric_D_prod(const Layout& L, const double* a, const double* b, int d, int i, int j, int k) {
  if (L.closed[d]) {
    const long long base = line_base(L, d, i, j, k), s = L.es[d];
    return appc_D([&](int m) { return a[base + m * s] * b[base + m * s]; }, line_pos(d, i, j, k), L.n[d]);
  }
  return stencil_D_prod(a, b, eidx(L, i, j, k), L.es[d]);
}

// interface value at i+1/2 along d of the cell field f (Sec. 7 step 3), App. C on a closed axis
GBR_HD double metric_I(const Layout& L, const double* f, int d, int i, int j, int k) {
  if (L.closed[d]) {
    const long long base = line_base(L, d, i, j, k), s = L.es[d];
    int c[3] = {i, j, k};
    return appc_face([&](int m) { return f[base + m * s]; }, c[d], L.n[d]);
  }
  return stencil_I(f, eidx(L, i, j, k), L.es[d]);
}

// Eq. (GCL_metrics) (3D) or its z = zeta reduction (2D), Eq. (Jac-matrix),
// unhatted metrics (viscous) and Sec. 4 time metrics (moving).
// mh_given: the 3D hat metrics are already in G.mh (the MIG4 line kernels formed them)
GBR_HD void body_metrics(const GeoArgs& G, int i, int j, int k, bool mh_given = false) {
  const Layout& L = G.L;
  const long long EC = L.ecount;
  const long long e = eidx(L, i, j, k);
  const int nd = L.nd;
  double m[3][3];
  double det;
  if (nd == 3 && mh_given) {
    for (int ee = 0; ee < 3; ++ee)
      for (int a = 0; a < 3; ++a) m[ee][a] = G.mh[(ee * 3 + a) * EC + e];
  } else if (nd == 3) {
    for (int ee = 0; ee < 3; ++ee) {
      const int f = (ee + 1) % 3, g = (ee + 2) % 3;
      for (int a = 0; a < 3; ++a) {
        const int b = (a + 1) % 3, c = (a + 2) % 3;
        // e.g. xi^_x = (y_eta z)_zeta - (y_zeta z)_eta
        const double t1 = metric_D_prod(L, G.xd + (b * 3 + f) * EC, G.xc + c * EC, g, i, j, k);
        const double t2 = metric_D_prod(L, G.xd + (b * 3 + g) * EC, G.xc + c * EC, f, i, j, k);
        m[ee][a] = t1 - t2;
      }
    }
  }
  if (nd == 3) {
    const double xx = G.xd[0 * EC + e], xe = G.xd[1 * EC + e], xz = G.xd[2 * EC + e];
    const double yx = G.xd[3 * EC + e], ye = G.xd[4 * EC + e], yz = G.xd[5 * EC + e];
    const double zx = G.xd[6 * EC + e], ze = G.xd[7 * EC + e], zz = G.xd[8 * EC + e];
    det = xx * (ye * zz - ze * yz) - yx * (xe * zz - ze * xz) + zx * (xe * yz - ye * xz);
  } else {
    const double xx = G.xd[0 * EC + e], xe = G.xd[1 * EC + e];
    const double yx = G.xd[3 * EC + e], ye = G.xd[4 * EC + e];
    m[0][0] = ye;
    m[0][1] = -xe;
    m[1][0] = -yx;
    m[1][1] = xx;
    det = xx * ye - xe * yx;
  }
  for (int ee = 0; ee < nd; ++ee)
    for (int a = 0; a < nd; ++a) G.mh[(ee * 3 + a) * EC + e] = m[ee][a];
  G.det[e] = det;
  if (G.viscous) {
    const double idet = 1.0 / det;
    for (int ee = 0; ee < nd; ++ee)
      for (int a = 0; a < nd; ++a) G.mu[(ee * 3 + a) * EC + e] = m[ee][a] * idet;
  }
  if (G.moving) {
    for (int ee = 0; ee < nd; ++ee) {
      double s = 0.0;
      for (int a = 0; a < nd; ++a) s = gfma(G.vc[a * EC + e], m[ee][a], s);
      G.mt[ee * EC + e] = -s;
    }
  }
}

// Interface geometry the FP64 interface stages would otherwise form at every stage from fh and fu
// (functions of the mesh alone), stored per interface in fg: the unit normal nu = n^/|n^|, |n^|^2,
// 1/|n^|, |n^|, 1/|n^|^2 and, viscous, m_e = sum_b (d xi_e/d x_b) n^_b (the chain rule contracted
// with n^, Sec. 5.2).  Each value is formed by the same operations in the same order as the
// FP32 interface stages form them in place (face_unlimited, hllc, face_flux): the stored values
// equal what the stages would form.
enum { FG_NU = 0, FG_NN2 = 3, FG_INN = 4, FG_NN = 5, FG_INN2 = 6, FG_M = 7, FG_COUNT = 10 };
inline int fg_count(bool viscous) { return viscous ? FG_COUNT : FG_M; }

GBR_HD void body_face_geo(const GeoArgs& G, double* fg, int d, int i, int j, int k) {
  const Layout& L = G.L;
  const int nd = L.nd;
  const long long FC = L.fcount[d], f = fidx(L, d, i, j, k);
  double nh[3] = {0.0, 0.0, 0.0}, nn2 = 0.0;
  for (int a = 0; a < nd; ++a) {
    nh[a] = G.fh[d][a * FC + f];
    nn2 = gfma(nh[a], nh[a], nn2);
  }
  const double inn = grsqrt(nn2);
  for (int a = 0; a < 3; ++a) fg[(FG_NU + a) * FC + f] = nh[a] * inn;
  fg[FG_NN2 * FC + f] = nn2;
  fg[FG_INN * FC + f] = inn;
  fg[FG_NN * FC + f] = nn2 * inn;
  fg[FG_INN2 * FC + f] = inn * inn;
  if (G.viscous)
    for (int e = 0; e < nd; ++e) {
      const double* fu = G.fu[d] + (e * nd) * FC + f;
      double acc = fu[0] * nh[0];
      for (int b = 1; b < nd; ++b) acc = gfma(fu[b * FC], nh[b], acc);
      fg[(FG_M + e) * FC + f] = acc;
    }
}

// Sec. 7 step 3: interface values of whole metric products, interface i+1/2 along d
GBR_HD void body_face_metrics(const GeoArgs& G, int d, int i, int j, int k) {
  const Layout& L = G.L;
  const long long EC = L.ecount, FC = L.fcount[d];
  const long long e = eidx(L, i, j, k), s = L.es[d];
  const long long f = fidx(L, d, i, j, k);
  const int nd = L.nd;
  (void)e;
  (void)s;
  for (int a = 0; a < nd; ++a) G.fh[d][a * FC + f] = metric_I(L, G.mh + (d * 3 + a) * EC, d, i, j, k);
  if (G.viscous)
    for (int ee = 0; ee < nd; ++ee)
      for (int a = 0; a < nd; ++a) G.fu[d][(ee * nd + a) * FC + f] = metric_I(L, G.mu + (ee * 3 + a) * EC, d, i, j, k);
  if (G.moving) G.ft[d][f] = metric_I(L, G.mt + d * EC, d, i, j, k);
}

// Eq. (Jacb2) with the same interface difference as the flux divergence; J for the update
GBR_HD void body_gcl(const GeoArgs& G, int i, int j, int k) {
  const Layout& L = G.L;
  const long long c = cidx(L, i, j, k);
  if (G.moving) {
    double s = 0.0;
    for (int d = 0; d < L.nd; ++d) {
      const long long fhi = fidx(L, d, i, j, k);
      s = s + (G.ft[d][fhi] - G.ft[d][fhi - L.fs[d][d]]);
    }
    G.gcl[c] = -s;
  }
  G.jac[c] = 1.0 / G.det[eidx(L, i, j, k)];
}

// Sec. 8.2 motion families evaluated at extended node index (i, j, k)
struct Motion {
  double origin[3], h[3], amp[3], omega, k[3][3];
};
GBR_HD void body_motion(const Layout& L, const Motion& M, double st, double ct, double* nodes, double* nvel, int i,
                        int j, int k) {
  const int m[3] = {i, j, k};
  const long long id = nidx(L, i, j, k);
  for (int a = 0; a < L.nd; ++a) {
    double S = 1.0;
    for (int b = 0; b < L.nd; ++b)
      if (M.k[a][b] != 0.0) S *= sin(M.k[a][b] * (m[b] * M.h[b]));
    nodes[a * L.ncount + id] = M.origin[a] + m[a] * M.h[a] + M.amp[a] * st * S;
    nvel[a * L.ncount + id] = M.amp[a] * ct * S;
  }
}

// ---------------------------------------------------------------------------
// Right-hand-side bodies (Sec. 3, Sec. 5)
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// Right-hand side bodies, templated on the compute type R of the reconstruction:
// R = double is the FP64 path; R = float is the mixed path, where primitives,
// gradients, characteristic reconstruction, limiter, Riemann and viscous fluxes
// run and are stored in FP32, while the conserved state, the metrics and 1/J
// (computed in FP64 by the geometry bodies), the GCL term, the flux divergence
// and the RK accumulation stay FP64.  Every literal in the templated bodies is
// written as R(...) so that the float path does no FP64 arithmetic.
// ---------------------------------------------------------------------------
template <class R>
struct PhysR {
  R gamma, gm1, igm1;
  R mu_ref, suth_s, it_ref;
  R alpha_d;                 // alpha^D
  R mp_alpha, mp_beta, mp_eps;
  R kfac;
  // The first derivatives are stored as K f' (K = kE6Scale with E6 gradients, 1 with IG4), and
  // the constants that multiply them carry 1/K: gh = 1/(2K) (f'/2 of the unlimited states and of
  // the alpha-damping states), sd = 1/(24 K) (the f' part of f''/12), alpha_k = K alpha^D (the
  // damped interface gradients are kept in units of K f'), hk = 1/(2K) and tk = -1/(3K) (mu/2
  // and lambda/2 per unit of mu on those gradients)
  R gh, sd, alpha_k, hk, tk;
  R hmu_ref, tmu_ref, hmk_ref;  // hk mu_ref, tk mu_ref, hk mu_ref kfac (constant viscosity)
  int sutherland;
};
template <class R>
inline PhysR<R> phys_r(const Phys& ph, double K) {
  PhysR<R> r;
  r.gamma = R(ph.gamma);
  r.gm1 = R(ph.gm1);
  r.igm1 = R(ph.igm1);
  r.mu_ref = R(ph.mu_ref);
  r.suth_s = R(ph.suth_s);
  r.it_ref = R(ph.it_ref);
  r.alpha_d = R(ph.alpha_d);
  r.mp_alpha = R(ph.mp_alpha);
  r.mp_beta = R(ph.mp_beta);
  r.mp_eps = R(ph.mp_eps);
  r.kfac = R(ph.kfac);
  r.gh = R(0.5 / K);
  r.sd = R(1.0 / (24.0 * K));
  r.alpha_k = R(ph.alpha_d * K);
  r.hk = R(0.5 / K);
  r.tk = R(-1.0 / (3.0 * K));
  r.hmu_ref = r.hk * r.mu_ref;  // the products face_flux forms from mu, in the path's type
  r.tmu_ref = r.tk * r.mu_ref;
  r.hmk_ref = r.hmu_ref * r.kfac;
  r.sutherland = ph.sutherland;
  return r;
}

template <class R>
struct RhsArgsT {
  Layout L;
  Phys ph;
  PhysR<R> pr;
  const double* q;      // [nv][ncells] conserved state of the stage
  R* prim;              // [nv][pcount] primitives with halo; the pressure slot holds p - pref
  double pref;          // pressure offset of the stored primitives (mixed path; 0 on the FP64 path)
  R pref_r;             // the same in the path's type (the mixed path's offset is an FP32 number)
  R* temp;              // [pcount] T = p/rho (viscous)
  R* g1[3];             // [nv (+1 T)][pcount] first derivatives along d
  R* g2[3];             // [nv][pcount] second derivatives along d, as f'' / 12 (second_deriv_12)
  const R* fh[3];       // [nd][fcount] hat metrics n^ at interfaces (FP32 copies on the mixed path)
  const R* fu[3];       // [nd][nd][fcount] unhatted metrics d xi_e / d x_a at interfaces
  const R* ft[3];       // [fcount] hat xi_t at interfaces (moving)
  const R* fg[3];       // [FG_COUNT][fcount] interface geometry derived from fh, fu (FP64 path; body_face_geo)
  R* flux[3];           // [nv][fcount] F^ - F^v at interfaces
  const double* inflow; // [nv][nk][nj]
  int bc[3][2];
  int viscous;
};
using RhsArgs = RhsArgsT<double>;

// single-precision helpers of the mixed path (plain compares: FP32 min/max are cheap)
GBR_HD float grsqrt(float x) {
#ifdef __CUDA_ARCH__
  return rsqrtf(x);
#else
  return 1.0f / std::sqrt(x);
#endif
}
GBR_HD float gfma(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return fmaf(a, b, c);
#else
  return a * b + c;
#endif
}
GBR_HD bool is_pos(float x) { return x > 0.0f; }
GBR_HD bool is_neg(float x) { return x < 0.0f; }
GBR_HD float gmin(float a, float b) { return a < b ? a : b; }
GBR_HD float gmax(float a, float b) { return a > b ? a : b; }
GBR_HD float gabs(float x) { return x < 0.0f ? -x : x; }
GBR_HD float minmod(float a, float b) {  // App. E
  if (a > 0.0f && b > 0.0f) return a < b ? a : b;
  if (a < 0.0f && b < 0.0f) return a > b ? a : b;
  return 0.0f;
}
GBR_HD float gsqrt(float x) {
#ifdef __CUDA_ARCH__
  return sqrtf(x);
#else
  return std::sqrt(x);
#endif
}
GBR_HD double gsqrt(double x) { return sqrt(x); }

// E6 first derivative (Eq. E6_grads, read with differences)
// Sixty times the E6 first derivative: 45 d1 - 9 d2 + d3 with d_m = f_{i+m} - f_{i-m}, five
// operations against six for 3/4 d1 - 3/20 d2 + 1/60 d3; the stored first derivatives carry this
// factor (kE6Scale) and their users fold 1/60 into constants they multiply by anyway (PhysR)
constexpr double kE6Scale = 60.0;
template <class R>
GBR_HD R stencil_E6x60(const R* f, long long e, long long s) {
  return gfma(R(45), f[e + s] - f[e - s], gfma(R(-9), f[e + 2 * s] - f[e - 2 * s], f[e + 3 * s] - f[e - 3 * s]));
}

// Sec. 2: primitives P = [rho, u.., p] (and T = p/rho, R = 1) of state cell c stored at padded
// index p, evaluated in the path's type R from the FP64 state (the mixed path rounds the state
// to FP32 first: the stored primitives are FP32 either way, and the FP64 divide is what would
// bound this pass)
// The pressure is stored as p - pref: on the mixed path pref is a pressure of the flow (set with
// the state), so that FP32 keeps the digits of the pressure differences; the energy offset
// pref/(gamma-1) is taken off in FP64 before the rounding.  pref = 0 on the FP64 path.
// dq (mixed path, or null): the FP32 increment of the stage state over q, Q_s = q + dq (the
// stage states of a step are kept as Q^n plus an FP32 increment, see body_update); added after
// the rounding to FP32.
// The stored pressures carry p - pref, and pref = 0 on the FP64 path
template <class R>
constexpr bool kPrefZero = sizeof(R) == sizeof(double);
template <int ND, class R>
GBR_HD void prim_store(const RhsArgsT<R>& A, const double* q, const float* dq, long long c, long long p) {
  constexpr int NV = ND + 2;
  const Layout& L = A.L;
  const long long NC = L.ncells, PC = L.pcount;
  const R rho = dq ? R(q[c]) + R(dq[c]) : R(q[c]);
  const R ir = grcp(rho);
  R ke = R(0);
  A.prim[p] = rho;
  for (int a = 0; a < ND; ++a) {
    const long long o = (1 + a) * NC + c;
    const R m = dq ? R(q[o]) + R(dq[o]) : R(q[o]);
    const R u = m * ir;
    A.prim[(1 + a) * PC + p] = u;
    ke = gfma(m, u, ke);
  }
  const long long oE = (NV - 1) * NC + c;
  // E - pref/(gamma - 1) (pref = 0 on the FP64 path: nothing to subtract)
  const double Eoff = kPrefZero<R> ? q[oE] : q[oE] - A.pref * A.ph.igm1;
  const R Erel = dq ? R(Eoff) + R(dq[oE]) : R(Eoff);
  const R prel = A.pr.gm1 * (Erel - R(0.5) * ke);  // p - pref
  A.prim[(NV - 1) * PC + p] = prel;
  if (A.viscous) A.temp[p] = (kPrefZero<R> ? prel : prel + A.pref_r) * ir;
}

// primitives at interior cells
template <int ND, class R>
GBR_HD void body_prim(const RhsArgsT<R>& A, int i, int j, int k) {
  prim_store<ND>(A, A.q, nullptr, cidx(A.L, i, j, k), pidx(A.L, i, j, k));
}

// Primitives on the whole padded box in one pass (interior and ghost layers): a ghost cell takes
// the primitives of its source cell found axis by axis -- periodic wrap, zero-gradient clamp,
// slip-wall mirror, or the x-low inflow data -- which is exactly what the axis-by-axis ghost
// copies of body_halo produce (corners included), with the same arithmetic per value.  A slip
// wall mirrors cell g - 1 into ghost layer g and reflects the velocity about the
// unit normal of the wall interface; several walls reflect in axis order, each normal taken at
// the cross-section the axis-by-axis filling sees (earlier axes' coordinates clamped to the
// cells, later axes' at the source cell).
// SPECIAL = false: no inflow or wall boundary on this grid (every ghost cell is a periodic or
// zero-gradient copy), so the FP64 ghost path is left out of the instantiation (registers)
template <int ND, class R, bool SPECIAL = true>
GBR_HD void body_prim_halo(const RhsArgsT<R>& A, const double* q, const float* dq, int i, int j, int k) {
  constexpr int NV = ND + 2;
  const Layout& L = A.L;
  int c[3] = {i, j, k};
  const int own[3] = {i, j, k};
  bool inflow = false;
  int wall[3] = {0, 0, 0};
  #pragma unroll
  for (int a = 0; a < ND; ++a) {
    const int n = L.n[a];
    if (c[a] < 0) {
      if (L.per[a]) {
        c[a] += n;
      } else if (a == 0 && A.bc[0][0] == 2) {
        inflow = true;
        c[a] = 0;
      } else if (A.bc[a][0] == 3) {
        wall[a] = -1;
        c[a] = -c[a] - 1;
      } else {
        c[a] = 0;
      }
    } else if (c[a] >= n) {
      if (L.per[a]) {
        c[a] -= n;
      } else if (A.bc[a][1] == 3) {
        wall[a] = 1;
        c[a] = 2 * n - 1 - c[a];
      } else {
        c[a] = n - 1;
      }
    }
  }
  const long long p = pidx(L, i, j, k);
  const long long PC = L.pcount;
  if (!SPECIAL || (!inflow && !(wall[0] | wall[1] | wall[2]))) {
    prim_store<ND>(A, q, dq, cidx(L, c[0], c[1], c[2]), p);
    return;
  }
  // the source state in FP64
  double rho, u[3] = {0.0, 0.0, 0.0}, pr;
  if (inflow) {
    const long long plane = (long long)L.n[1] * L.n[2];
    const long long ib = (long long)c[2] * L.n[1] + c[1];
    rho = A.inflow[ib];
    for (int a = 0; a < ND; ++a) u[a] = A.inflow[(1 + a) * plane + ib];
    pr = A.inflow[(NV - 1) * plane + ib];
  } else {
    const long long cs = cidx(L, c[0], c[1], c[2]), NC = L.ncells;
    auto qv = [&](int v) { return dq ? q[v * NC + cs] + (double)dq[v * NC + cs] : q[v * NC + cs]; };
    rho = qv(0);
    const double ir = 1.0 / rho;
    double ke = 0.0;
    for (int a = 0; a < ND; ++a) {
      const double m = qv(1 + a);
      u[a] = m * ir;
      ke = gfma(m, u[a], ke);
    }
    pr = A.ph.gm1 * (qv(NV - 1) - 0.5 * ke);
  }
  #pragma unroll
  for (int a = 0; a < ND; ++a) {
    if (!wall[a]) continue;
    int fc[3];
    for (int b = 0; b < 3; ++b) {
      if (b < a) fc[b] = own[b] < 0 ? 0 : (own[b] >= L.n[b] ? L.n[b] - 1 : own[b]);
      else fc[b] = c[b];
    }
    fc[a] = wall[a] < 0 ? -1 : L.n[a] - 1;  // the wall interface
    const long long FC = L.fcount[a], f = fidx(L, a, fc[0], fc[1], fc[2]);
    double nh[3] = {0.0, 0.0, 0.0}, nn = 0.0;
    for (int b = 0; b < ND; ++b) {
      nh[b] = A.fh[a][b * FC + f];
      nn = gfma(nh[b], nh[b], nn);
    }
    const double inv = 1.0 / sqrt(nn);
    double un = 0.0;
    for (int b = 0; b < ND; ++b) {
      nh[b] *= inv;
      un = gfma(u[b], nh[b], un);
    }
    for (int b = 0; b < ND; ++b) u[b] = gfma(-2.0 * un, nh[b], u[b]);
  }
  A.prim[p] = R(rho);
  for (int a = 0; a < ND; ++a) A.prim[(1 + a) * PC + p] = R(u[a]);
  A.prim[(NV - 1) * PC + p] = R(pr - A.pref);
  if (A.viscous) A.temp[p] = R(pr / rho);
}

// ghost layers along axis d for the cross-section cell (i, j, k) (coordinate d ignored):
// periodic copy, zero gradient, or Dirichlet inflow on the x-low side
template <int ND, class R>
GBR_HD void body_halo(const RhsArgsT<R>& A, int d, int i, int j, int k) {
  constexpr int NV = ND + 2;
  const Layout& L = A.L;
  const long long PC = L.pcount, s = L.ps[d];
  int c0[3] = {i, j, k};
  c0[d] = 0;
  const long long base = pidx(L, c0[0], c0[1], c0[2]);  // cell 0 along d
  const int n = L.n[d];
  const int nf = NV + (A.viscous ? 1 : 0);
  for (int f = 0; f < nf; ++f) {
    R* F = (f < NV) ? A.prim + f * PC : A.temp;
    for (int g = 1; g <= H; ++g) {
      const long long lo = base - g * s, hi = base + (n - 1 + g) * s;
      if (L.per[d]) {
        F[lo] = F[base + (n - g) * s];
        F[hi] = F[base + (g - 1) * s];
      } else {
        if (A.bc[d][0] == 2) {
          const long long ib = ((long long)k * L.n[1] + j);
          if (f < NV) {
            F[lo] = R(A.inflow[f * L.n[1] * L.n[2] + ib]);
          } else {
            F[lo] = R(A.inflow[(NV - 1) * L.n[1] * L.n[2] + ib] / A.inflow[ib]);
          }
        } else {
          F[lo] = F[base];
        }
        F[hi] = F[base + (n - 1) * s];
      }
    }
  }
}

// Sec. 5.1 step 1: E6 first derivatives along e (primitives and T)
template <int ND, class R>
GBR_HD void body_grad1(const RhsArgsT<R>& A, int e, int i, int j, int k) {
  constexpr int NV = ND + 2;
  const Layout& L = A.L;
  const long long PC = L.pcount, p = pidx(L, i, j, k), s = L.ps[e];
  for (int c = 0; c < NV; ++c) A.g1[e][c * PC + p] = stencil_E6x60(A.prim + c * PC, p, s);
  if (A.viscous) A.g1[e][NV * PC + p] = stencil_E6x60(A.temp, p, s);
}

// Sec. 5.1 step 1: f''_i = 2 (f_{i+1} - 2 f_i + f_{i-1}) - 0.5 (f'_{i+1} - f'_{i-1}), kept as
// f''_i / 12: the scale at which the unlimited states use it (Eq. legendre_polys: f'/2 + f''/12,
// one fused multiply-add per field instead of a multiply and one) and at which the App. E
// curvatures d = W'' enter the bounds (mp_bound folds the factor 12 into constants it multiplies
// anyway).  The FP32 path forms it inside the interface kernel (from f and f' of the four cells
// of the stencil, which it loads anyway): no array and no pass.  The FP64 path stores it once per
// cell and direction, which costs fewer FP64 operations than forming it twice per interface.
template <class R>
constexpr bool kFaceFormsG2 = sizeof(R) == sizeof(float);
// The FP64 interface stages read the mesh-only interface geometry from fg (body_face_geo); the FP32
// ones, issue-bound, form it (fewer instructions than the loads and their addresses)
template <class R>
constexpr bool kFaceGeo = sizeof(R) == sizeof(double);

// f1 holds K f' (PhysR): sd = 1/(24 K)
template <class R, class I>
GBR_HD R second_deriv_12(const R* f, const R* f1, I p, I s, R sd) {
  if constexpr (sizeof(R) == sizeof(double)) {
    // FP64 (pipe-bound pass): five operations, (f_{i+1} - 2 f_i + f_{i-1}) / 6 as one fused
    // multiply-add on -(f'_{i+1} - f'_{i-1}) / 24
    const R c2 = gfma(R(-2), f[p], f[p + s]) + f[p - s];
    return gfma(R(1.0 / 6.0), c2, -sd * (f1[p + s] - f1[p - s]));
  } else {
    // FP32 (inside the interface kernel, where the form above measured 1.3 % slower)
    return R(1.0 / 6.0) * (f[p + s] - R(2) * f[p] + f[p - s]) - sd * (f1[p + s] - f1[p - s]);
  }
}

template <int ND, class R>
GBR_HD void body_grad2(const RhsArgsT<R>& A, int e, int i, int j, int k) {
  constexpr int NV = ND + 2;
  const Layout& L = A.L;
  const long long PC = L.pcount, p = pidx(L, i, j, k), s = L.ps[e];
  for (int c = 0; c < NV; ++c) {
    const R* f = A.prim + c * PC;
    const R* f1 = A.g1[e] + c * PC;
    A.g2[e][c * PC + p] = second_deriv_12(f, f1, p, s, A.pr.sd);
  }
}

// ---------------------------------------------------------------------------
// MIG4 (Eq. IG4_grads, alpha = 5/14): alpha f'_{i-1} + f'_i + alpha f'_{i+1} =
// (2 + alpha)/3 (f_{i+1} - f_{i-1}) + (4 alpha - 1)/12 (f_{i+2} - f_{i-2}).
// The matrix is the same for every line of a direction, so its Thomas factors
// are computed once (on the device, ig4_factor) and each line is one forward and
// one backward sweep.  Periodic axis: the cyclic system over the n cells by the
// Sherman-Morrison formula (gamma = -1: first diagonal 2, last 1 + alpha^2,
// correction vector z solved once); open axis: the padded line of n + 2H cells
// whose three end points at each side take explicit rows (second-order
// one-sided, fourth-order biased, fourth-order central).
// Table layout per direction (doubles): periodic: cp[n], inv[n], z[n], kinv, P[n];
// open: cp[m], inv[m] with m = n + 2H.
// ---------------------------------------------------------------------------

inline long long ig4_table_len(int n, bool periodic) { return periodic ? 4LL * n + 1 : 2LL * (n + 2 * H); }

GBR_HD void ig4_factor(double* t, int n, bool periodic) {
  const double al = kIg4Alpha;
  if (periodic) {
    double* cp = t;
    double* inv = t + n;
    double* z = t + 2 * n;
    // modified diagonal: b_0 = 1 - gamma = 2, b_{n-1} = 1 - alpha^2 / gamma = 1 + alpha^2
    double den = 2.0;
    inv[0] = 1.0 / den;
    cp[0] = al * inv[0];
    for (int i = 1; i < n; ++i) {
      const double b = (i == n - 1) ? 1.0 + al * al : 1.0;
      const double c = (i == n - 1) ? 0.0 : al;
      den = b - al * cp[i - 1];
      inv[i] = 1.0 / den;
      cp[i] = c * inv[i];
    }
    // z = T'^-1 u, u = (gamma, 0, .., 0, alpha)
    z[0] = -1.0 * inv[0];
    for (int i = 1; i < n; ++i) z[i] = ((i == n - 1 ? al : 0.0) - al * z[i - 1]) * inv[i];
    for (int i = n - 2; i >= 0; --i) z[i] -= cp[i] * z[i + 1];
    // x = y - (y_0 - alpha y_{n-1}) / (1 + z_0 - alpha z_{n-1}) z   (v = (1, 0, .., 0, alpha / gamma))
    t[3 * n] = 1.0 / (1.0 + z[0] - al * z[n - 1]);
    // weights of y_0 in the forward results: y_0 = sum_k P_k g_k, P_k = prod_{j<k} (-cp_j), so that
    // y_0 (and the correction factor) is known before the backward sweep (ig4_solve)
    double* P = t + 3 * n + 1;
    P[0] = 1.0;
    for (int i = 1; i < n; ++i) P[i] = -cp[i - 1] * P[i - 1];
  } else {
    const int m = n + 2 * H;
    double* cp = t;
    double* inv = t + m;
    for (int i = 0; i < m; ++i) {
      const bool expl = i < 3 || i >= m - 3;
      const double a = expl ? 0.0 : al, c = expl ? 0.0 : al;
      const double den = 1.0 - (i > 0 ? a * cp[i - 1] : 0.0);
      inv[i] = 1.0 / den;
      cp[i] = c * inv[i];
    }
  }
}

// IG4 right side of row i from the values f_{i-2} .. f_{i+2} (stride s)
template <class R>
GBR_HD R ig4_rhs(const R* f, long long p, long long s) {
  return R((2.0 + kIg4Alpha) / 3.0) * (f[p + s] - f[p - s]) + R((4.0 * kIg4Alpha - 1.0) / 12.0) * (f[p + 2 * s] - f[p - 2 * s]);
}

// IG4 right side of a row from the window values f_{i-2}, f_{i-1}, f_{i+1}, f_{i+2} (the same
// arithmetic as ig4_rhs)
template <class R>
GBR_HD R ig4_rhs_w(R fm2, R fm1, R fp1, R fp2) {
  return R((2.0 + kIg4Alpha) / 3.0) * (fp1 - fm1) + R((4.0 * kIg4Alpha - 1.0) / 12.0) * (fp2 - fm2);
}

// One IG4 line.  f: cell 0 of the line, w: cell 0 of a work column (may be f itself: in place),
// both with distance S between cells; out: cell -H of the destination, distance so.  The forward
// sweep reads each f into a register window before w is written at or below it, and also sums
// y_0 = sum_k P_k g_k (periodic), so the Sherman-Morrison factor is known before the backward
// sweep, which then forms each final value once and stores it (and the periodic images) at
// out + (c + H) so for cell c; out may alias w (each row is read before it is overwritten).
// In place on a periodic line (out aliasing w) the correction pass reads row m before it
// writes it and writes images only at rows it has read or never reads.
// Periodic: the n cells with the images of f at -2, -1, n, n + 1; the derivative at 0 .. n-1 and
// its images at -3 .. -1 and n .. n+2.  Open: the padded line -H .. n+H-1.  y_0 is the backward
// sweep's own end value summed in another order.
// FP32 sums y_0 in the forward sweep (one pass less over the column); FP64, whose line solves are
// bound by the FP64 pipe, does not spend the extra multiply-add per cell and forms y_0 by the
// backward sweep in the work column before the correction.
template <class R>
constexpr bool kIg4SumY0 = sizeof(R) == sizeof(float);

template <class R>
GBR_HD void ig4_solve(const R* t, int n, bool periodic, const R* f, R* w, long long S, R* out, long long so) {
  const R al = R(kIg4Alpha);
  if (periodic) {
    const R* cp = t;
    const R* inv = t + n;
    const R* z = t + 2 * n;
    const R* P = t + 3 * n + 1;
    R w0 = f[-2 * S], w1 = f[-S], w2 = f[0], w3 = f[S], w4 = f[2 * S];
    R prev = R(0), y0 = R(0);
    for (int m = 0; m < n; ++m) {
      const R r = ig4_rhs_w(w0, w1, w3, w4);
      prev = (m == 0) ? r * inv[0] : (r - al * prev) * inv[m];
      if constexpr (kIg4SumY0<R>) y0 = y0 + P[m] * prev;
      w0 = w1;
      w1 = w2;
      w2 = w3;
      w3 = w4;
      if (m + 1 < n) w4 = f[(m + 3) * S];
      w[m * S] = prev;
    }
    R y = prev;
    if constexpr (kIg4SumY0<R>) {
      const R fac = (y0 - al * prev) * t[3 * n];
      for (int m = n - 1; m >= 0; --m) {
        if (m < n - 1) y = w[m * S] - cp[m] * y;
        const R x = y - fac * z[m];
        out[(m + H) * so] = x;
        if (m >= n - 3) out[(m - n + H) * so] = x;  // images -3 .. -1
        if (m <= 2) out[(m + n + H) * so] = x;      // images n .. n + 2
      }
    } else {
      // backward sweep and correction in the work column, then the rows out (when out is not w)
      for (int m = n - 2; m >= 0; --m) {
        y = w[m * S] - cp[m] * y;
        w[m * S] = y;
      }
      const R fac = (y - al * w[(n - 1) * S]) * t[3 * n];
      for (int m = 0; m < n; ++m) w[m * S] = w[m * S] - fac * z[m];
      for (int m = 1; m <= 3; ++m) {  // periodic images of the derivative the gradient box needs
        w[-m * S] = w[(n - m) * S];
        w[(n - 1 + m) * S] = w[(m - 1) * S];
      }
      if (out != w - H * S)
        for (int c = -3; c < n + 3; ++c) out[(c + H) * so] = w[c * S];
    }
  } else {
    const int M = n + 2 * H;
    const R* cp = t;
    const R* inv = t + M;
    const R* f0 = f - H * S;  // padded cell -H: row 0
    R* w0r = w - H * S;
    R w0 = R(0), w1 = R(0), w2 = R(0), w3 = f0[0], w4 = f0[S], w5 = f0[2 * S], w6 = f0[3 * S];
    R prev = R(0);
    for (int m = 0; m < M; ++m) {
      R r;
      if (m == 0) r = R(-1.5) * w3 + R(2) * w4 - R(0.5) * w5;
      else if (m == 1) r = R(-0.25) * w2 - R(5.0 / 6.0) * w3 + R(1.5) * w4 - R(0.5) * w5 + w6 * R(1.0 / 12.0);
      else if (m == 2 || m == M - 3) r = R(2.0 / 3.0) * (w4 - w2) - (w5 - w1) * R(1.0 / 12.0);
      else if (m == M - 2) r = R(0.25) * w4 + R(5.0 / 6.0) * w3 - R(1.5) * w2 + R(0.5) * w1 - w0 * R(1.0 / 12.0);
      else if (m == M - 1) r = R(1.5) * w3 - R(2) * w2 + R(0.5) * w1;
      else r = ig4_rhs_w(w1, w2, w4, w5);
      const bool expl = m < 3 || m >= M - 3;
      prev = (m == 0 || expl) ? r * inv[m] : (r - al * prev) * inv[m];
      w0 = w1;
      w1 = w2;
      w2 = w3;
      w3 = w4;
      w4 = w5;
      w5 = w6;
      if (m + 4 < M) w6 = f0[(m + 4) * S];
      w0r[m * S] = prev;
    }
    R y = prev;
    out[(M - 1) * so] = y;
    for (int m = M - 2; m >= 0; --m) {
      y = w0r[m * S] - cp[m] * y;
      out[m * so] = y;
    }
  }
}

// One line of f' along e through padded cell (i, j, k) (coordinate e ignored): field f, output g
template <class R>
GBR_HD void ig4_line(const Layout& L, const R* t, int e, const R* f, R* g, int i, int j, int k) {
  int c0[3] = {i, j, k};
  c0[e] = 0;
  const long long base = pidx(L, c0[0], c0[1], c0[2]);  // cell 0 of the line
  const long long s = L.ps[e];
  ig4_solve(t, L.n[e], L.per[e] != 0, f + base, g + base, s, g + base - H * s, s);
}

// Both derivatives along e in one pass over the first-derivative box: f' at the cell (stored),
// and, inside the second-derivative box `b2`, f'' from f' of the two neighbours recomputed with
// the same stencil -- the values are those of body_grad1 followed by body_grad2.
template <int ND, class R>
GBR_HD void body_grad12(const RhsArgsT<R>& A, int e, const Box& b2, int i, int j, int k) {
  constexpr int NV = ND + 2;
  const Layout& L = A.L;
  const long long PC = L.pcount, p = pidx(L, i, j, k), s = L.ps[e];
  const bool second = i >= b2.lo[0] && i < b2.hi[0] && j >= b2.lo[1] && j < b2.hi[1] && k >= b2.lo[2] &&
                      k < b2.hi[2];
  for (int c = 0; c < NV; ++c) {
    const R* f = A.prim + c * PC;
    A.g1[e][c * PC + p] = stencil_E6x60(f, p, s);
    if (second) {
      const R f1p = stencil_E6x60(f, p + s, s), f1m = stencil_E6x60(f, p - s, s);
      A.g2[e][c * PC + p] = gfma(R(1.0 / 6.0), gfma(R(-2), f[p], f[p + s]) + f[p - s], -A.pr.sd * (f1p - f1m));  // as second_deriv_12
    }
  }
  if (A.viscous) A.g1[e][NV * PC + p] = stencil_E6x60(A.temp, p, s);
}

// App. A projection x -> R^{-1} x for the face eigenvectors (unit normal nu,
// face rho*a = ra and a^2).  Row order: U - a, U (x2 or x3), U + a.
template <int ND, class R>
GBR_HD void project(const R* nu, R ra, R a2, const R* x, R* W) {
  if (ND == 3) {
    // rows U -/+ a: x_p -/+ (rho a) s, each one fused multiply-add
    const R s = gfma(nu[0], x[1], gfma(nu[1], x[2], nu[2] * x[3]));
    const R e = gfma(a2, x[0], -x[4]);
    W[0] = gfma(-ra, s, x[4]);
    W[1] = gfma(nu[0], e, gfma(nu[1], x[3], -nu[2] * x[2]));
    W[2] = gfma(nu[2], e, gfma(nu[0], x[2], -nu[1] * x[1]));
    W[3] = gfma(-nu[1], e, gfma(nu[0], x[3], -nu[2] * x[1]));
    W[4] = gfma(ra, s, x[4]);
  } else {
    const R s = gfma(nu[0], x[1], nu[1] * x[2]);
    W[0] = gfma(-ra, s, x[3]);
    W[1] = gfma(a2, x[0], -x[3]);
    W[2] = gfma(nu[0], x[2], -nu[1] * x[1]);
    W[3] = gfma(ra, s, x[3]);
  }
}

// App. A back-projection onto a base state: out = base + R d (hira = 1 / (2 rho a)); the base
// enters as the addend of each row's innermost fused multiply-add
template <int ND, class R>
GBR_HD void back_project(const R* nu, R hira, R ia2, const R* dl, const R* base, R* out) {
  if (ND == 3) {
    const R s04 = dl[0] + dl[4];
    const R q = (dl[4] - dl[0]) * hira;
    const R x = gfma(nu[0], dl[1], gfma(nu[2], dl[2], -nu[1] * dl[3]));
    out[0] = gfma(ia2, gfma(R(0.5), s04, x), base[0]);
    out[1] = gfma(nu[0], q, gfma(-nu[1], dl[2], gfma(-nu[2], dl[3], base[1])));
    out[2] = gfma(nu[1], q, gfma(-nu[2], dl[1], gfma(nu[0], dl[2], base[2])));
    out[3] = gfma(nu[2], q, gfma(nu[1], dl[1], gfma(nu[0], dl[3], base[3])));
    out[4] = gfma(R(0.5), s04, base[4]);
  } else {
    const R s03 = dl[0] + dl[3];
    const R q = (dl[3] - dl[0]) * hira;
    out[0] = gfma(ia2, gfma(R(0.5), s03, dl[1]), base[0]);
    out[1] = gfma(nu[0], q, gfma(-nu[1], dl[2], base[1]));
    out[2] = gfma(nu[1], q, gfma(nu[0], dl[2], base[2]));
    out[3] = gfma(R(0.5), s03, base[3]);
  }
}

// App. E limiter written relative to the base cell value W_base:
//   f  = W_face - W_base,  dm = W_base - W_up,  dp = W_down - W_base,
//   du, db, dd = curvatures d / 12 of the up, base and down cells (the scale of the stored f''),
//   so that W^MD - W_base = (dp - 12 d^M) / 2 and W^LC - W_base = 16 d^M + dm / 2.
// mp_keep is the test (W^L - W_base)(W^L - W^MP) <= eps that leaves the state
// unchanged; mp_bound returns the limited W_face - W_base when it fails.
// FP64: the products and sums are FP64; every comparison, min, max, minmod and
// the median work on the bit patterns (integer pipe) and select one of their
// arguments exactly.
GBR_HD bool mp_keep(double f, double dm, double dp, const PhysR<double>& ph) {
  const long long bf = dbits(f);
  const long long bmp = bminmod(dbits(dp), dbits(ph.mp_beta * dm));  // W^MP - W_base
  // exactly non-positive product when f lies between 0 and W^MP - W_base
  const long long kf = bkey(bf), km = bkey(bmp), ke = okey(ph.mp_eps);
  const bool between = (km >= 0) ? (kf >= 0 && kf <= km) : (kf <= 0 && kf >= km);
  return (between && ke >= 0) || okey(f * (f - bitsd(bmp))) <= ke;
}
GBR_HD double mp_bound(double f, double dm, double dp, double du, double db, double dd, const PhysR<double>& ph) {
  const double dmp = bitsd(bminmod(dbits(db), dbits(dd)));  // d^M_{i+1/2}
  const double dmm = bitsd(bminmod(dbits(du), dbits(db)));  // d^M_{i-1/2}
  const long long bdp = dbits(dp), bf = dbits(f);
  const long long md = dbits(gfma(-6.0, dmp, 0.5 * dp));       // W^MD - W_base
  const long long ul = dbits(ph.mp_alpha * dm);                // W^UL - W_base
  const long long lc = dbits(gfma(16.0, dmm, 0.5 * dm));       // W^LC - W_base
  // W^min, W^max relative to W_base (W_base itself maps to 0)
  const long long lo = bmax(bmin(bmin(0LL, bdp), md), bmin(bmin(0LL, ul), lc));
  const long long hi = bmin(bmax(bmax(0LL, bdp), md), bmax(bmax(0LL, ul), lc));
  // W^L + minmod(W^min - W^L, W^max - W^L) is the median of (W^L, W^min, W^max)
  return bitsd(bmax(bmin(bf, lo), bmin(bmax(bf, lo), hi)));
}
// FP32 (mixed path): the same steps with plain single-precision compares
GBR_HD bool mp_keep(float f, float dm, float dp, const PhysR<float>& ph) {
  const float mmp = minmod(dp, ph.mp_beta * dm);
  return f * (f - mmp) <= ph.mp_eps;
}
GBR_HD float mp_bound(float f, float dm, float dp, float du, float db, float dd, const PhysR<float>& ph) {
  const float dmp = minmod(db, dd);
  const float dmm = minmod(du, db);
  const float md = gfma(-6.0f, dmp, 0.5f * dp);
  const float ul = ph.mp_alpha * dm;
  const float lc = gfma(16.0f, dmm, 0.5f * dm);
  const float lo = gmax(gmin(gmin(0.0f, dp), md), gmin(gmin(0.0f, ul), lc));
  const float hi = gmin(gmax(gmax(0.0f, dp), md), gmax(gmax(0.0f, ul), lc));
  return gmax(gmin(f, lo), gmin(gmax(f, lo), hi));
}

// Sec. 5.1.1 HLLC with grid motion; P = [rho, u.., p]
// The states carry p - pref (pref = 0 on the FP64 path): the absolute pressure enters the sound
// speeds, the energy and the energy flux; the pressure difference of S* and the momentum flux's
// pressure term use p - pref (the dropped pref n^ has zero divergence by the metric identities).
template <int ND, bool MOV, class R>
GBR_HD void hllc(const R* PL, const R* PR, const R* nh, R nn2, R nn, R inn2, R nt, const PhysR<R>& ph, R pref, R* F) {
  constexpr int NV = ND + 2;
  // left and right states (kept in scalars: no runtime-indexed arrays)
  const R rl = PL[0], rr = PR[0];
  const R dpl = PL[NV - 1], dpr = PR[NV - 1];
  const R pl = kPrefZero<R> ? dpl : dpl + pref, pr = kPrefZero<R> ? dpr : dpr + pref;
  // t = 1/sqrt(gamma p rho) = 1/(rho c): c = gamma p t and 1/rho = gamma p t^2, no division
  const R gpl = ph.gamma * pl, gpr = ph.gamma * pr;
  const R tl = grsqrt(gpl * rl), tr = grsqrt(gpr * rr);
  R q2l = R(0), q2r = R(0), Ul = nt, Ur = nt;
  #pragma unroll
  for (int a = 0; a < ND; ++a) {
    q2l = gfma(PL[1 + a], PL[1 + a], q2l);
    q2r = gfma(PR[1 + a], PR[1 + a], q2r);
    Ul = gfma(nh[a], PL[1 + a], Ul);  // contravariant velocity, Sec. 2
    Ur = gfma(nh[a], PR[1 + a], Ur);
  }
  const R El = gfma(pl, ph.igm1, R(0.5) * rl * q2l), Er = gfma(pr, ph.igm1, R(0.5) * rr * q2r);
  // speeds of sound c = sqrt(gamma p / rho) = |gamma p| t: the absolute value keeps the formula's
  // value for a reconstructed state whose density and pressure are both negative (the App. E bounds
  // do not exclude one at a sawtooth of cell values)
  const R cl = gabs(gpl) * tl, cr = gabs(gpr) * tr;
  const R SL = gmin(gfma(-cl, nn, Ul), gfma(-cr, nn, Ur));
  const R SR = gmax(gfma(cl, nn, Ul), gfma(cr, nn, Ur));
  const R aL = rl * (SL - Ul), aR = rr * (SR - Ur);
  const R Ss = gdiv(aR * Ur - aL * Ul + (dpl - dpr) * nn2, aR - aL);
  // branches of Sec. 5.1.1: S^L >= 0 -> F^L; S^L < 0 <= S* -> F*L; S* < 0 < S^R -> F*R; else F^R
  const bool left = !is_neg(SL) || !is_neg(Ss);
  const bool star = is_neg(SL) && (left || is_pos(SR));
  const R rs = left ? rl : rr, ps = left ? pl : pr, dps = left ? dpl : dpr;
  const R Us = left ? Ul : Ur, Es = left ? El : Er, S = left ? SL : SR;
  R us[ND];
  #pragma unroll
  for (int a = 0; a < ND; ++a) us[a] = left ? PL[1 + a] : PR[1 + a];
  // The mass and momentum fluxes of the chosen branch, F^K or F^K + S (Q*K - QK), grouped by
  // what they multiply: rho k1 and rho u_a k1 + n^_a k2, with k1 = U and k2 = p - pref outside the
  // star region and k1 = U + S dg, k2 = p - pref + S fw inside it (dg, fw below)
  R k1 = Us, k2 = dps;
  R Fe;
  if constexpr (MOV) Fe = gfma(Es + ps, Us, -nt * ps);
  else Fe = (Es + ps) * Us;  // xi_t = 0
  if (star) {
    // Q*K = rho (S - U)/(S - S*) [1, u + n^ (S* - U)/|n^|^2, E/rho + (S* - U)((S* - xi_t)/|n^|^2 + p/(rho (S - U)))]
    // The correction S (Q*K - QK) is formed with the factor (S* - U) taken out,
    //   Q*K - QK = (S* - U)/(S - S*) [rho, rho u, E] + rho (S - U)/(S - S*) (S* - U) [0, n^/|n^|^2, (S* - xi_t)/|n^|^2 + p/(rho (S - U))],
    // instead of as a difference of two O(rho) states multiplied by S ~ c: at low Mach numbers the
    // difference would lose a factor c/|U| of the working precision.
    const R rA = rs * (S - Us);
    const R B = S - Ss;
    const R inv = grcp(rA * B);
    const R g = rA * inv;             // 1 / (S - S*)
    const R fac = rA * g;             // rho (S - U) / (S - S*)
    const R p_rA = ps * B * inv;      // p / (rho (S - U))
    const R dS = Ss - Us;
    const R dg = dS * g;              // (S* - U) / (S - S*)
    const R fw = fac * dS * inn2;
    k1 = gfma(S, dg, Us);
    k2 = gfma(S, fw, dps);
    Fe = gfma(S * dS, gfma(fac, gfma(MOV ? Ss - nt : Ss, inn2, p_rA), Es * g), Fe);
  }
  F[0] = rs * k1;
  #pragma unroll
  for (int a = 0; a < ND; ++a) F[1 + a] = gfma(rs * us[a], k1, nh[a] * k2);
  F[NV - 1] = Fe;
}

// One interface i+1/2 along d: Sec. 5.1 steps 2-6 and Sec. 5.2 steps 1-4, in three stages so
// that the kernel can hand the limiter's bound work of a whole block to as few warps as possible:
// face_unlimited (face state, projected differences, unlimited states, the App. E test),
// face_bounds (the curvatures' projection and the bounds of the fields that failed the test),
// face_flux (back-projection, HLLC, viscous flux, store).
// The characteristic quantities are formed from projected differences of neighbouring cells
// and the limited states are returned relative to the base cell (P^L = P_i + R dW_L), which is
// the same arithmetic as projecting the cell values themselves, in a different rounding order.
template <int ND, class R>
struct FaceCtx {
  static constexpr int NV = ND + 2;
  FaceIx<R> p1, f;      // padded index of cell i, interface index
  R nh[ND], nu[ND];     // n^ and the unit normal
  R nn2, inn, nt;       // |n^|^2, 1/|n^| (formed on the FP32 path only; FP64 reads fg), hat xi_t
  R ra, a2, hira, ia2;  // face state of the eigenvectors (hira = 1 / (2 rho a))
  R Wd[3][NV];          // projected differences of cells i-1 .. i+2
  R dL[NV], dR[NV];     // W^L - W_i, W^R - W_{i+1}
  unsigned limit;       // bit c: left field c fails the App. E test; bit NV + c: right
};

// DD: the sweep direction fixed at compile time (0 .. 2; the single-solver kernels, one launch per
// direction), or -1 for d given at run time (the batch, whose launches mix directions)
template <int ND, bool MOV, class R, int DD = -1>
GBR_HD void face_unlimited(const RhsArgsT<R>& A, int d_in, int i, int j, int k, FaceCtx<ND, R>& C) {
  constexpr int NV = ND + 2;
  const int d = DD >= 0 ? DD : d_in;
  const Layout& L = A.L;
  const PhysR<R>& ph = A.pr;
  using I = FaceIx<R>;
  const I PC = (I)L.pcount, s = DD == 0 ? I(1) : (I)L.ps[d];
  const I p1 = face_pidx<I>(L, i, j, k);
  const I pp[4] = {p1 - s, p1, p1 + s, p1 + 2 * s};
  const I FC = (I)L.fcount[d];
  const I f = face_fidx<I>(L, d, i, j, k);
  const R* P = A.prim;
  C.p1 = p1;
  C.f = f;
  #pragma unroll
  for (int a = 0; a < ND; ++a) C.nh[a] = R(A.fh[d][a * FC + f]);
  C.nt = MOV ? R(A.ft[d][f]) : R(0);
  if constexpr (kFaceGeo<R>) {
    // FP64: |n^|^2 and the unit normal from the stored interface geometry
    const R* g = A.fg[d] + f;
    C.nn2 = g[FG_NN2 * FC];
    #pragma unroll
    for (int a = 0; a < ND; ++a) C.nu[a] = g[(FG_NU + a) * FC];
  } else {
    R nn2 = R(0);
    #pragma unroll
    for (int a = 0; a < ND; ++a) nn2 = gfma(C.nh[a], C.nh[a], nn2);
    C.nn2 = nn2;
    C.inn = grsqrt(nn2);
    #pragma unroll
    for (int a = 0; a < ND; ++a) C.nu[a] = C.nh[a] * C.inn;
  }
  // face state of the eigenvectors: mean of rho and p of cells i, i+1, kept doubled
  // (rb2 = 2 rho-bar, pb2 = 2 p-bar: the halvings fold into powers of two below)
  const R rb2 = P[pp[1]] + P[pp[2]];
  const R psum = P[(NV - 1) * PC + pp[1]] + P[(NV - 1) * PC + pp[2]];
  const R pb2 = kPrefZero<R> ? psum : psum + R(2) * A.pref_r;
  // a = sqrt(gamma p / rho): with t = 1/sqrt(gamma p rho), rho a = gamma p rho t, 1/(rho a) = t,
  // a = gamma p t and 1/a = rho t -- one reciprocal square root, no division.  From the doubled
  // state: g4 = 4 gamma p rho and t2 = 1/sqrt(g4) = t/2 (exact scalings by powers of two), so
  // 1/(2 rho a) = t2, rho a = g4 t2 / 2, a = (2 gamma p) t2 and 1/a = (2 rho) t2.
  const R gp2 = ph.gamma * pb2;
  const R g4 = gp2 * rb2;
  const R t2 = grsqrt(g4);
  C.hira = t2;
  C.ra = R(0.5) * (g4 * t2);
  const R a_ = gp2 * t2;
  C.a2 = a_ * a_;
  const R ia = rb2 * t2;
  C.ia2 = ia * ia;
  // projected differences dW = R^-1 (P_{m+1} - P_m) of the four cells i-1 .. i+2
  #pragma unroll
  for (int m = 0; m < 3; ++m) {
    R x[NV];
    #pragma unroll
    for (int c = 0; c < NV; ++c) x[c] = P[c * PC + pp[m + 1]] - P[c * PC + pp[m]];
    project<ND>(C.nu, C.ra, C.a2, x, C.Wd[m]);
  }
  // Eq. (legendre_polys) unlimited states relative to the base cells, projected
  // after combining: W^L - W_i = R^-1 (f'_i / 2 + f''_i / 12),
  // W^R - W_{i+1} = R^-1 (-f'_{i+1} / 2 + f''_{i+1} / 12)
  if constexpr (kFaceFormsG2<R>) {
    // FP32: f'' of cells i and i+1 formed here (the same formula as body_grad2) from the
    // primitives and f' of cells i-1 .. i+2 -- two loads of f' per field instead of two of f''
    R xl[NV], xr[NV];
    #pragma unroll
    for (int c = 0; c < NV; ++c) {
      const R* f = P + c * PC;
      const R* f1 = A.g1[d] + c * PC;
      xl[c] = gfma(ph.gh, f1[pp[1]], second_deriv_12(f, f1, pp[1], s, ph.sd));
      xr[c] = gfma(-ph.gh, f1[pp[2]], second_deriv_12(f, f1, pp[2], s, ph.sd));
    }
    project<ND>(C.nu, C.ra, C.a2, xl, C.dL);
    project<ND>(C.nu, C.ra, C.a2, xr, C.dR);
  } else {
    R x[NV];
    #pragma unroll
    for (int c = 0; c < NV; ++c)
      x[c] = gfma(ph.gh, A.g1[d][c * PC + pp[1]], A.g2[d][c * PC + pp[1]]);
    project<ND>(C.nu, C.ra, C.a2, x, C.dL);
    #pragma unroll
    for (int c = 0; c < NV; ++c)
      x[c] = gfma(-ph.gh, A.g1[d][c * PC + pp[2]], A.g2[d][c * PC + pp[2]]);
    project<ND>(C.nu, C.ra, C.a2, x, C.dR);
  }
  // App. E test per field and side
  unsigned limit = 0;
  #pragma unroll
  for (int c = 0; c < NV; ++c) {
    limit |= mp_keep(C.dL[c], C.Wd[0][c], C.Wd[1][c], ph) ? 0u : (1u << c);
    limit |= mp_keep(C.dR[c], -C.Wd[2][c], -C.Wd[1][c], ph) ? 0u : (1u << (NV + c));
  }
  C.limit = limit;
}

// App. E bounds of the fields that failed the test: the curvatures d / 12 of cells i-1 .. i+2 are
// projected with the face's eigenvectors (only here), then each failing state is limited.
// FP32 forms the four f'' here (keeping those of cells i and i+1 from face_unlimited instead
// measured 3 % slower: more live registers); FP64 reads them from the f'' array.
template <int ND, class R, int DD = -1>
GBR_HD void face_bounds(const RhsArgsT<R>& A, int d_in, const R* nu, R ra, R a2, FaceIx<R> p1, unsigned limit,
                        const R (*Wd)[ND + 2], R* dL, R* dR) {
  constexpr int NV = ND + 2;
  const int d = DD >= 0 ? DD : d_in;
  const Layout& L = A.L;
  using I = FaceIx<R>;
  const I PC = (I)L.pcount, s = DD == 0 ? I(1) : (I)L.ps[d];
  const I pp[4] = {p1 - s, p1, p1 + s, p1 + 2 * s};
  R W2[4][NV];
  #pragma unroll
  for (int m = 0; m < 4; ++m) {
    R x[NV];
    #pragma unroll
    for (int c = 0; c < NV; ++c) {
      if constexpr (kFaceFormsG2<R>)
        x[c] = second_deriv_12(A.prim + c * PC, A.g1[d] + c * PC, pp[m], s, A.pr.sd);
      else
        x[c] = A.g2[d][c * PC + pp[m]];
    }
    project<ND>(nu, ra, a2, x, W2[m]);
  }
  #pragma unroll
  for (int c = 0; c < NV; ++c) {
    if (limit & (1u << c)) dL[c] = mp_bound(dL[c], Wd[0][c], Wd[1][c], W2[0][c], W2[1][c], W2[2][c], A.pr);
    if (limit & (1u << (NV + c))) dR[c] = mp_bound(dR[c], -Wd[2][c], -Wd[1][c], W2[3][c], W2[2][c], W2[1][c], A.pr);
  }
}

template <int ND, bool VISC, bool MOV, class R, int DD = -1>
GBR_HD void face_flux(const RhsArgsT<R>& A, int d_in, int i, int j, int k, const FaceCtx<ND, R>& C) {
  constexpr int NV = ND + 2;
  const int d = DD >= 0 ? DD : d_in;
  const Layout& L = A.L;
  const PhysR<R>& ph = A.pr;
  using I = FaceIx<R>;
  const I PC = (I)L.pcount, s = DD == 0 ? I(1) : (I)L.ps[d];
  const I p1 = C.p1;
  const I pp[4] = {p1 - s, p1, p1 + s, p1 + 2 * s};
  const I FC = (I)L.fcount[d];
  const I f = C.f;
  const R* P = A.prim;
  const R* nh = C.nh;
  const R nn2 = C.nn2, nt = C.nt;
  R nn, inn2;  // |n^| and 1/|n^|^2
  if constexpr (kFaceGeo<R>) {
    nn = A.fg[d][FG_NN * FC + f];
    inn2 = A.fg[d][FG_INN2 * FC + f];
  } else {
    nn = nn2 * C.inn;
    inn2 = C.inn * C.inn;
  }
  R PL[NV], PR[NV];
  {
    R B1[NV], B2[NV];  // the base cells i, i+1
    #pragma unroll
    for (int c = 0; c < NV; ++c) {
      B1[c] = P[c * PC + pp[1]];
      B2[c] = P[c * PC + pp[2]];
    }
    back_project<ND>(C.nu, C.hira, C.ia2, C.dL, B1, PL);
    back_project<ND>(C.nu, C.hira, C.ia2, C.dR, B2, PR);
  }
  R F[NV];
  hllc<ND, MOV>(PL, PR, nh, nn2, nn, inn2, nt, ph, A.pref_r, F);

  if (VISC) {
    // Sec. 5.2 alpha-damping on [u.., T].  gc2[v][e] = 2 K d(phi_v)/d(xi_e) at the interface (the
    // stored derivatives carry K, PhysR): Eq. (AD-eqn1) along the sweep, the sum of the two cells'
    // gradients across it (reading: the paper is silent on them); the factor 1/(2K) is folded
    // into mu, lambda and kappa below (hk, tk).
    R gc2[ND + 1][ND];
    R phs[ND + 1];  // phi^L + phi^R = 2 x the interface value of [u.., T]
    #pragma unroll
    for (int v = 0; v <= ND; ++v) {
      const R* val = (v < ND) ? P + (1 + v) * PC : A.temp;
      const int gi = (v < ND) ? (1 + v) : NV;
      const R gd1 = A.g1[d][gi * PC + pp[1]], gd2 = A.g1[d][gi * PC + pp[2]];
      const R phiL = gfma(ph.gh, gd1, val[pp[1]]);   // Eq. (AD-eqn2), beta^D = 0 (gd: K f')
      const R phiR = gfma(-ph.gh, gd2, val[pp[2]]);
      #pragma unroll
      for (int e = 0; e < ND; ++e) {
        if (e == d) {
          gc2[v][e] = gfma(ph.alpha_k, phiR - phiL, gd1 + gd2);  // 2 K x Eq. (AD-eqn1)
        } else {
          gc2[v][e] = A.g1[e][gi * PC + pp[1]] + A.g1[e][gi * PC + pp[2]];
        }
      }
      phs[v] = phiL + phiR;
    }
    // The flux needs only tau n^ and beta . n^ (Eq. shear-str, thermal-work), so the chain rule
    // d/dx_a = sum_e (d xi_e/d x_a) d/d xi_e (Eq. AD-eqn3) is contracted with n^ first:
    //   m_e = sum_b xi_e,x_b n^_b,  s_e = sum_b n^_b du_b/d xi_e,
    //   (grad u n^)_a = sum_e m_e du_a/dxi_e,  (grad u^T n^)_a = sum_e xi_e,x_a s_e,
    //   div u = sum_a sum_e xi_e,x_a du_a/dxi_e,  grad T . n^ = sum_e m_e dT/dxi_e,
    //   beta . n^ = kappa grad T . n^ + u . (tau n^)   (tau symmetric)
    const R* fu = A.fu[d];
    R xe[ND][ND];  // xe[e][a] = d xi_e / d x_a at the interface
    #pragma unroll
    for (int e = 0; e < ND; ++e)
      #pragma unroll
      for (int a = 0; a < ND; ++a) xe[e][a] = R(fu[(e * ND + a) * FC + f]);
    R m[ND], sv[ND];
    #pragma unroll
    for (int e = 0; e < ND; ++e) {
      R acc = xe[e][0] * nh[0], acs = nh[0] * gc2[0][e];
      #pragma unroll
      for (int b = 1; b < ND; ++b) {
        if constexpr (!kFaceGeo<R>) acc = gfma(xe[e][b], nh[b], acc);
        acs = gfma(nh[b], gc2[b][e], acs);
      }
      if constexpr (kFaceGeo<R>) acc = A.fg[d][(FG_M + e) * FC + f];  // stored (body_face_geo)
      m[e] = acc;
      sv[e] = acs;
    }
    // mu / 2, -mu / 3 (lambda / 2) and mu kfac / 2: constants unless mu follows Sutherland's law
    R hmu = ph.hmu_ref, tmu = ph.tmu_ref, hmk = ph.hmk_ref;
    if (ph.sutherland) {
      const R th = R(0.5) * phs[ND] * ph.it_ref;
      const R mu = ph.mu_ref * (th * gsqrt(th)) * ((R(1) + ph.suth_s) / (th + ph.suth_s));
      hmu = ph.hk * mu;
      tmu = ph.tk * mu;
      hmk = hmu * ph.kfac;
    }
    R div2 = R(0);
    #pragma unroll
    for (int a = 0; a < ND; ++a)
      #pragma unroll
      for (int e = 0; e < ND; ++e) div2 = gfma(xe[e][a], gc2[a][e], div2);
    const R hlamdiv = tmu * div2;  // lambda div u / 2, lambda = -2/3 mu
    R bn = R(0);  // 2 beta . n^ minus its conduction part
    #pragma unroll
    for (int a = 0; a < ND; ++a) {
      R t12 = R(0);  // (grad u n^)_a + (grad u^T n^)_a, one chain
      #pragma unroll
      for (int e = 0; e < ND; ++e) {
        t12 = gfma(m[e], gc2[a][e], t12);
        t12 = gfma(xe[e][a], sv[e], t12);
      }
      const R taun = gfma(hmu, t12, hlamdiv * nh[a]);  // (tau n^)_a
      F[1 + a] -= taun;
      bn = gfma(phs[a], taun, bn);  // 2 u . (tau n^)
    }
    R gTn = R(0);
    #pragma unroll
    for (int e = 0; e < ND; ++e) gTn = gfma(m[e], gc2[ND][e], gTn);
    F[NV - 1] -= gfma(hmk, gTn, R(0.5) * bn);
  }
  #pragma unroll
  for (int c = 0; c < NV; ++c) A.flux[d][c * FC + f] = F[c];
}

// the whole interface in one thread (host emulation)
template <int ND, bool VISC, bool MOV, class R>
GBR_HD void body_face(const RhsArgsT<R>& A, int d, int i, int j, int k) {
  FaceCtx<ND, R> C;
  face_unlimited<ND, MOV>(A, d, i, j, k, C);
  if (C.limit) face_bounds<ND>(A, d, C.nu, C.ra, C.a2, C.p1, C.limit, C.Wd, C.dL, C.dR);
  face_flux<ND, VISC, MOV>(A, d, i, j, k, C);
}

// Sec. 3 divergence, Sec. 4 time split, App. B stage combination (FP64; the
// interface fluxes are read in the path's type R and accumulated in FP64).
template <class R>
struct UpdArgsT {
  Layout L;
  const R* flux[3];
  const double* qs;     // state of this stage
  const double* q0;     // Q^n
  double* out;          // new state (mode 1) or L(Q) (mode 0)
  const double* jac;
  const float* jac32;   // mixed path: FP32 copy of J (else null)
  const double* gcl;
  const double* sigma;  // sponge (or null)
  double qamb[5];
  const double* dt;     // device scalar
  double ca, cb, cc;    // out = ca q0 + cb qs + cc dt L
  int mode;             // 0: out = L, 1: RK combination
  // mixed path, static mesh, no sponge: the stage states as Q^n + FP32 increments (or null)
  const float* dq_in;   // increment of this stage's state (null in the first stage)
  float* dq_out;        // increment of the next stage's state (null in the last stage: out = Q^n+1)
};
using UpdArgs = UpdArgsT<double>;

// |x| > 1.79e308 (overflow or NaN) and x <= 0 tested on the bit pattern (integer pipe; the
// FP64 pipe is the scarce one on this GPU)
constexpr long long kUpdHuge = 0x7FEFDCF158ADBB99LL;  // bit pattern of 1.79e308
GBR_HD bool upd_not_finite(double x) { return (dbits(x) & kMag) > kUpdHuge; }
GBR_HD bool upd_not_positive(double x) { return dbits(x) <= 0; }  // +0, negatives, -0
GBR_HD bool upd_not_finite_f(float x) {  // |x| above the largest float: infinity or NaN
#ifdef __CUDA_ARCH__
  return (__float_as_uint(x) & 0x7FFFFFFFu) > 0x7F7FFFFFu;
#else
  unsigned b;
  std::memcpy(&b, &x, sizeof b);
  return (b & 0x7FFFFFFFu) > 0x7F7FFFFFu;
#endif
}

// -sum_d (F_{i+1/2} - F_{i-1/2}) of component v, written (F_lo - F_hi) + ... so the first term
// needs no subtraction from zero: the same rounding as 0 - (F_hi - F_lo) - ..., one operation fewer
template <int ND, class R>
GBR_HD R upd_flux_sum(const UpdArgsT<R>& U, int v, int i, int j, int k) {
  const Layout& L = U.L;
  R r = R(0);
  #pragma unroll
  for (int d = 0; d < ND; ++d) {
    const long long fhi = fidx(L, d, i, j, k);
    const long long FC = L.fcount[d];
    const R t = U.flux[d][v * FC + fhi - L.fs[d][d]] - U.flux[d][v * FC + fhi];
    r = (d == 0) ? t : r + t;
  }
  return r;
}

// SP: the launch may carry a sponge (false: U.sigma is null for every cell it updates; the FP32
// increment loop then has no sponge path, which costs registers at 32 per thread)
template <int ND, bool MOV, class R, bool SP = true>
GBR_HD bool body_update(const UpdArgsT<R>& U, int i, int j, int k) {
  constexpr int NV = ND + 2;
  const Layout& L = U.L;
  const long long c = cidx(L, i, j, k), NC = L.ncells;
  bool bad = false;
  // RK combination out = ca q0 + cb qs + cc dt J r with r the residual: dt cc J is one factor per
  // cell; the first SSP-RK3 stage (qs = q0, ca + cb = 1) is out = qs + dt J r and reads Q^n once
  const bool first = U.qs == U.q0 && U.ca + U.cb == 1.0;
  if constexpr (sizeof(R) == sizeof(float) && !MOV) {
    // mixed path, static mesh, no sponge: the increment dt cc J r is formed in FP32 (r is an FP32
    // sum; its relative error stays that of r) and only the state combination is FP64
    if (U.mode == 1 && U.jac32 && (U.dq_in || U.dq_out)) {
      // SSP-RK3 with ca + cb = 1 in increments: Q_s = Q^n + D_s, D_1 = dt L_0,
      // D_2 = 1/4 D_1 + 1/4 dt L_1, Q^n+1 = Q^n + 2/3 D_2 + 2/3 dt L_2, each D in FP32 (its size
      // is that of the step's change, far below Q), one FP64 addition per value and step;
      // L = J r - sigma (Q_s - Q_amb) with the sponge
      const float dtJf = float((*U.dt) * U.cc) * U.jac32[c];
      const float cbf = float(U.cb);
      // the sponge loop apart (a separate instantiation: the loop without it keeps its registers)
      auto stages = [&](auto sponge) {
        constexpr bool WS = decltype(sponge)::value;
        const double sg = WS ? U.sigma[c] : 0.0;
        const float dtsg = WS ? float((*U.dt) * U.cc * sg) : 0.0f;
        for (int v = 0; v < NV; ++v) {
          float dn = dtJf * upd_flux_sum<ND>(U, v, i, j, k);
          if constexpr (WS) {
            if (sg != 0.0) {
              float dev = float(U.q0[v * NC + c] - U.qamb[v]);
              if (U.dq_in) dev += U.dq_in[v * NC + c];
              dn = gfma(-dtsg, dev, dn);
            }
          }
          if (U.dq_in) dn = gfma(cbf, U.dq_in[v * NC + c], dn);
          if (U.dq_out) {
            U.dq_out[v * NC + c] = dn;
            bad |= upd_not_finite_f(dn);
          } else {
            const double o = U.q0[v * NC + c] + (double)dn;
            U.out[v * NC + c] = o;
            bad |= upd_not_finite(o) || (v == 0 && upd_not_positive(o));
          }
        }
      };
      if constexpr (SP) {
        if (U.sigma) stages(std::true_type{});
        else stages(std::false_type{});
      } else {
        stages(std::false_type{});
      }
      return bad;
    }
    if (U.mode == 1 && !U.sigma && U.jac32) {
      const float dtJf = float((*U.dt) * U.cc) * U.jac32[c];
      for (int v = 0; v < NV; ++v) {
        const R rsum = upd_flux_sum<ND>(U, v, i, j, k);
        const double inc = (double)(dtJf * rsum);
        const double qv = U.qs[v * NC + c];
        const double o = first ? qv + inc : gfma(U.ca, U.q0[v * NC + c], gfma(U.cb, qv, inc));
        U.out[v * NC + c] = o;
        bad |= upd_not_finite(o) || (v == 0 && upd_not_positive(o));
      }
      return bad;
    }
  }
  const double J = U.jac[c];
  const double dtJ = (U.mode == 1) ? (*U.dt) * U.cc * J : 0.0;
  for (int v = 0; v < NV; ++v) {
    // flux differences in the fluxes' own type (for neighbouring FP32 fluxes within a factor 2 of
    // each other the difference is exact), summed and converted to FP64 once
    R rsum = upd_flux_sum<ND>(U, v, i, j, k);
    const double res = (double)rsum;
    const double qv = U.qs[v * NC + c];
    const double r = MOV ? gfma(-U.gcl[c], qv, res) : res;  // residual before 1/J (GCL term, Eq. Jacb2)
    if (U.mode == 0 || U.sigma) {
      double Lv = J * r;
      if (U.sigma) Lv = gfma(-U.sigma[c], qv - U.qamb[v], Lv);
      if (U.mode == 0) {
        U.out[v * NC + c] = Lv;
        bad |= upd_not_finite(Lv);
        continue;
      }
      const double dtc = (*U.dt) * U.cc;
      const double o = gfma(U.ca, U.q0[v * NC + c], gfma(U.cb, qv, dtc * Lv));
      U.out[v * NC + c] = o;
      bad |= upd_not_finite(o) || (v == 0 && upd_not_positive(o));
      continue;
    }
    const double o = first ? gfma(dtJ, r, qv) : gfma(U.ca, U.q0[v * NC + c], gfma(U.cb, qv, dtJ * r));
    U.out[v * NC + c] = o;
    bad |= upd_not_finite(o) || (v == 0 && upd_not_positive(o));
  }
  return bad;
}

// App. B: per-cell min over directions of 1/(|U| + c |grad xi|), plus the
// viscous bound 1 / (nu_eff |grad xi|^2), nu_eff = max(4/3, gamma/Pr) mu / rho.
struct DtArgs {
  Layout L;
  Phys ph;
  const double* q;
  const double* mh;   // ext layout
  const double* mt;   // ext layout (moving) or null
  const double* jac;
  // mixed path: FP32 copies on the interior cells ([9][cells], [3][cells], [cells]; the FP32
  // time step then converts only the state), else null
  const float* mh32;
  const float* mt32;
  const float* jac32;
  // FP64 path on a static mesh: |grad xi_e| and |grad xi_e|^2 per direction ([2 nd][cells],
  // body_dt_geo), else null
  const double* gdt;
};

// The time step's metric norms on a static mesh, once per mesh: g2_e = sum_a (mh_ea J)^2 and
// sqrt(g2_e), by the operations and in the order of body_dt_r's own form (which then reads them
// instead): the stored values equal what it would form
GBR_HD void body_dt_geo(const DtArgs& D, double* gdt, int i, int j, int k) {
  const Layout& L = D.L;
  const int nd = L.nd;
  const long long c = cidx(L, i, j, k), NC = L.ncells, e = eidx(L, i, j, k), EC = L.ecount;
  const double J = D.jac[c];
  for (int ee = 0; ee < nd; ++ee) {
    double g2 = 0.0;
    for (int a = 0; a < nd; ++a) {
      const double m = D.mh[(ee * 3 + a) * EC + e] * J;
      g2 = gfma(m, m, g2);
    }
    gdt[ee * NC + c] = gsqrt(g2);
    gdt[(nd + ee) * NC + c] = g2;
  }
}

// FP32 copies of the cell metrics the mixed path's time step reads (interior cells)
GBR_HD void body_dt_f32(const DtArgs& D, float* mh32, float* mt32, float* jac32, int i, int j, int k) {
  const Layout& L = D.L;
  const long long c = cidx(L, i, j, k), NC = L.ncells, e = eidx(L, i, j, k), EC = L.ecount;
  for (int ee = 0; ee < L.nd; ++ee) {
    for (int a = 0; a < L.nd; ++a) mh32[(ee * 3 + a) * NC + c] = (float)D.mh[(ee * 3 + a) * EC + e];
    if (D.mt) mt32[ee * NC + c] = (float)D.mt[ee * EC + e];
  }
  jac32[c] = (float)D.jac[c];
}

// GS: the metric norms are read from D.gdt (FP64, static mesh; the instantiation chosen on the
// host); otherwise formed here (and read when D.gdt is set, a uniform run-time choice)
template <int ND, class R = double, bool GS = false>
GBR_HD R body_dt_r(const DtArgs& D, int i, int j, int k) {
  // evaluated in the path's type R (the mixed path's FP32 time step differs from the FP64 one by
  // FP32 round-off, far below the CFL number's own slack)
  constexpr int NV = ND + 2;
  const Layout& L = D.L;
  const Phys& ph = D.ph;
  const long long c = cidx(L, i, j, k), NC = L.ncells, e = eidx(L, i, j, k), EC = L.ecount;
  const R rho = R(D.q[c]);
  const R ir = grcp(rho);
  R u[ND], ke = R(0);
  for (int a = 0; a < ND; ++a) {
    const R m = R(D.q[(1 + a) * NC + c]);
    u[a] = m * ir;
    ke = gfma(m, u[a], ke);
  }
  const R pr = R(ph.gm1) * (R(D.q[(NV - 1) * NC + c]) - R(0.5) * ke);
  const R cs = gsqrt(R(ph.gamma) * pr * ir);
  constexpr bool F32 = sizeof(R) == sizeof(float);
  const R J = (F32 && D.jac32) ? R(D.jac32[c]) : R(D.jac[c]);
  R nu_eff = R(0);
  if (ph.viscous) {
    R mu = R(ph.mu_ref);
    if (ph.sutherland) {
      const R th = pr * ir * R(ph.it_ref);
      mu = R(ph.mu_ref) * (th * gsqrt(th)) * ((R(1) + R(ph.suth_s)) / (th + R(ph.suth_s)));
    }
    nu_eff = R(ph.dt_visc_fac) * mu * ir;
  }
  // min over directions of 1/(|U| + c |grad xi|) and 1/(nu_eff |grad xi|^2) as one division by the
  // largest denominator: division is correctly rounded and monotone, so the result is the same value
  R worst = R(0);
  const bool stored = GS || (!F32 && D.gdt != nullptr);
  for (int ee = 0; ee < ND; ++ee) {
    R Uc = D.mt ? ((F32 && D.mt32) ? R(D.mt32[ee * NC + c]) : R(D.mt[ee * EC + e])) * J : R(0);
    R g2 = R(0);
    for (int a = 0; a < ND; ++a) {
      const R mv = (F32 && D.mh32) ? R(D.mh32[(ee * 3 + a) * NC + c]) : R(D.mh[(ee * 3 + a) * EC + e]);
      const R m = mv * J;
      Uc = gfma(m, u[a], Uc);
      if (!stored) g2 = gfma(m, m, g2);
    }
    R gn;
    if (stored) {
      gn = R(D.gdt[ee * NC + c]);
      g2 = R(D.gdt[(ND + ee) * NC + c]);
    } else {
      gn = gsqrt(g2);
    }
    worst = gmax(worst, gabs(Uc) + cs * gn);
    if (ph.viscous) worst = gmax(worst, nu_eff * g2);
  }
  return R(1) / worst;  // +inf where nothing bounds the step
}

// the same as an FP64 number capped at 1e300 (the reduction's neutral value)
template <int ND, class R = double>
GBR_HD double body_dt(const DtArgs& D, int i, int j, int k) {
  return gmin(1.0e300, double(body_dt_r<ND, R>(D, i, j, k)));
}

}  // namespace gbr
