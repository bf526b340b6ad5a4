/*
 * TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously-correct FP64 CPU oracle of the per-RK-stage right-hand
 * side of arXiv 2303.10785: MEG6 gradient-based reconstruction with the improved
 * MP limiter, curvilinear HLLC, alpha-damping viscous flux, freestream-preserving
 * conservative metrics and the geometric-conservation term on moving meshes,
 * advanced by SSP-RK3.  Every function follows the paper's steps in the paper's
 * order; nothing is blocked, fused or reordered.  Only tests/, the smoke check
 * and bench.py's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant with the CUDA library in paper_2303_10785_b300/.
 *
 * Sections followed (paper numbering):
 *   Sec. 2   governing equations: fluxes, contravariant velocity, energy, stresses
 *   Sec. 3   conservative finite-difference residual Res
 *   Sec. 4   conservative metrics (Eq. GCL_metrics), time metrics, time split,
 *            Jacobian (Eq. Jac-matrix), (1/J)_t (Eq. Jacb2)
 *   Sec. 5.1 steps 1-7: E6 gradients (Eq. E6_grads), second derivative, projection
 *            (App. A eigenvectors), van Leer states (Eq. legendre_polys), improved MP
 *            limiter (App. E), back-projection, HLLC (Sec. 5.1.1), flux difference
 *   Sec. 5.2 alpha-damping viscous flux, steps 1-5
 *   Sec. 7   consistent metric derivative (Eq. FP-interp, FP-interp2) and
 *            interpolation (Eq. interp-formulae)
 *   App. B   SSP-RK3 and the CFL time step
 *   App. D   non-conservative metrics with the E4 derivative (negative control only)
 *
 * Where the paper is silent or garbled, the reading taken is stated beside the code that uses it.
 * Parity unpinned (oracle-to-GPU parity only): the face state used for the
 * eigenvectors, the MP-limiter constants alpha = beta = 4, the value of the
 * Sutherland constant S/T_ref of the jet, and the jet boundary/sponge forms.
 * (The time step, heat conduction and Sutherland's formula are pinned to closed
 * forms by tests/test_oracle_closures.py.)
 */
#include "orc.h"

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <string>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifdef ORC_COUNTING
#include "counting.h"
typedef CReal real;
OrcCounters orc_counters[8] = {};
int orc_phase = 0;
static inline real Sqrt(real a) { orc_counters[orc_phase].sqrt++; return CReal(std::sqrt(a.v)); }
#define ORC_PHASE(x) (orc_phase = (x))
static inline real Fabs(real a) { return CReal(std::fabs(a.v)); }
static inline double Dbl(real a) { return a.v; }
#else
typedef double real;
static inline real Sqrt(real a) { return std::sqrt(a); }
static inline real Fabs(real a) { return std::fabs(a); }
static inline double Dbl(real a) { return a; }
#define ORC_PHASE(x) ((void)0)
#endif
// phases of the counting build: 0 time step / RK combination, 1 primitives,
// 2 gradients, 3 interface fluxes, 4 divergence and source terms, 5 geometry
enum { PH_MISC = 0, PH_PRIM = 1, PH_GRAD = 2, PH_FACE = 3, PH_RES = 4, PH_GEOM = 5 };

static std::string g_err;
static int fail(const std::string& m) { g_err = m; return 1; }

static const int H = 6;   // ghost layers of the primitive state
static const int E = 10;  // geometry extension in cells beyond each side
// MIG4: geometry extension beyond each side of a periodic axis (IG4 on the unbounded
// unwrapped line, Sec. 7 step 2), and the margin kept to the ends of those lines for the
// cell metrics that are interpolated to interfaces
static const int kExtIG4 = 64;
static const int kCellIG4 = kExtIG4 - 10;

static inline real Min(real a, real b) { return (a < b) ? a : b; }
static inline real Max(real a, real b) { return (a > b) ? a : b; }
static inline real Min3(real a, real b, real c) { return Min(Min(a, b), c); }
static inline real Max3(real a, real b, real c) { return Max(Max(a, b), c); }
static inline real Sign(real a) { return (a > 0.0) ? real(1.0) : ((a < 0.0) ? real(-1.0) : real(0.0)); }
// App. E: minmod(a, b) = 1/2 (sign(a) + sign(b)) min(|a|, |b|)
static inline real minmod(real a, real b) { return 0.5 * (Sign(a) + Sign(b)) * Min(Fabs(a), Fabs(b)); }

// ---------------------------------------------------------------------------
// Boxes of cells and fields on them
// ---------------------------------------------------------------------------
struct Box {
  int lo[3], hi[3];  // inclusive lo, exclusive hi
  size_t size() const {
    return (size_t)(hi[0] - lo[0]) * (size_t)(hi[1] - lo[1]) * (size_t)(hi[2] - lo[2]);
  }
  size_t idx(int i, int j, int k) const {
    return ((size_t)(k - lo[2]) * (size_t)(hi[1] - lo[1]) + (size_t)(j - lo[1])) * (size_t)(hi[0] - lo[0]) +
           (size_t)(i - lo[0]);
  }
  bool has(int i, int j, int k) const {
    return i >= lo[0] && i < hi[0] && j >= lo[1] && j < hi[1] && k >= lo[2] && k < hi[2];
  }
  bool contains(const Box& o) const {
    for (int d = 0; d < 3; ++d)
      if (o.lo[d] < lo[d] || o.hi[d] > hi[d]) return false;
    return true;
  }
  Box grow(int d, int a, int b) const {
    Box r = *this;
    r.lo[d] -= a;
    r.hi[d] += b;
    return r;
  }
};

static Box box_and(const Box& a, const Box& b) {
  Box r;
  for (int d = 0; d < 3; ++d) {
    r.lo[d] = a.lo[d] > b.lo[d] ? a.lo[d] : b.lo[d];
    r.hi[d] = a.hi[d] < b.hi[d] ? a.hi[d] : b.hi[d];
  }
  return r;
}

struct Field {
  Box b;
  std::vector<real> v;
  Field() { b = Box{{0, 0, 0}, {0, 0, 0}}; }
  explicit Field(const Box& bb) : b(bb), v(bb.size(), real(0.0)) {}
#ifdef ORC_BOUNDS
  real& at(int i, int j, int k) {
    if (!b.has(i, j, k)) { std::fprintf(stderr, "orc: out of box %d %d %d\n", i, j, k); std::abort(); }
    return v[b.idx(i, j, k)];
  }
  real at(int i, int j, int k) const {
    if (!b.has(i, j, k)) { std::fprintf(stderr, "orc: out of box %d %d %d\n", i, j, k); std::abort(); }
    return v[b.idx(i, j, k)];
  }
#else
  real& at(int i, int j, int k) { return v[b.idx(i, j, k)]; }
  real at(int i, int j, int k) const { return v[b.idx(i, j, k)]; }
#endif
  // value shifted by s cells along axis d
  real sh(int i, int j, int k, int d, int s) const {
    int c[3] = {i, j, k};
    c[d] += s;
    return at(c[0], c[1], c[2]);
  }
};

#define FOR_BOX(B)                                              \
  _Pragma("omp parallel for collapse(2) schedule(static)")     \
  for (int k = (B).lo[2]; k < (B).hi[2]; ++k)                   \
    for (int j = (B).lo[1]; j < (B).hi[1]; ++j)                 \
      for (int i = (B).lo[0]; i < (B).hi[0]; ++i)

// ---------------------------------------------------------------------------
// One-dimensional operators along axis d (Sec. 5.1 step 1, Sec. 7, App. D)
// ---------------------------------------------------------------------------

// Eq. (E6_grads), read with differences:
// f'_i = 3/4 (f_{i+1} - f_{i-1}) - 3/20 (f_{i+2} - f_{i-2}) + 1/60 (f_{i+3} - f_{i-3})
static Field op_e6(const Field& f, int d) {
  Field o(f.b.grow(d, -3, -3));
  FOR_BOX(o.b) {
    o.at(i, j, k) = (3.0 / 4.0) * (f.sh(i, j, k, d, 1) - f.sh(i, j, k, d, -1)) -
                    (3.0 / 20.0) * (f.sh(i, j, k, d, 2) - f.sh(i, j, k, d, -2)) +
                    (1.0 / 60.0) * (f.sh(i, j, k, d, 3) - f.sh(i, j, k, d, -3));
  }
  return o;
}

// Eq. (4thorder-grads), App. D: f'_i = 2/3 (f_{i+1} - f_{i-1}) - 1/12 (f_{i+2} - f_{i-2})
static Field op_e4(const Field& f, int d) {
  Field o(f.b.grow(d, -2, -2));
  FOR_BOX(o.b) {
    o.at(i, j, k) = (2.0 / 3.0) * (f.sh(i, j, k, d, 1) - f.sh(i, j, k, d, -1)) -
                    (1.0 / 12.0) * (f.sh(i, j, k, d, 2) - f.sh(i, j, k, d, -2));
  }
  return o;
}

// Eq. (IG4_grads), read with differences, alpha = 5/14:
//   alpha f'_{i-1} + f'_i + alpha f'_{i+1} = (2 + alpha)/3 (f_{i+1} - f_{i-1}) + (4 alpha - 1)/12 (f_{i+2} - f_{i-2})
static const double kIG4Alpha = 5.0 / 14.0;

static real ig4_rhs(const real* f, int i) {
  const double a = kIG4Alpha;
  return (2.0 + a) / 3.0 * (f[i + 1] - f[i - 1]) + (4.0 * a - 1.0) / 12.0 * (f[i + 2] - f[i - 2]);
}

// Thomas algorithm for sub-diagonal a, diagonal b, super-diagonal c, right side r (length m);
// the first and last rows may be given with zero off-diagonals.
static void thomas(const std::vector<real>& a, const std::vector<real>& b, const std::vector<real>& c,
                   std::vector<real> r, std::vector<real>& x) {
  const int m = (int)b.size();
  std::vector<real> cp(m), rp(m);
  cp[0] = c[0] / b[0];
  rp[0] = r[0] / b[0];
  for (int i = 1; i < m; ++i) {
    const real den = b[i] - a[i] * cp[i - 1];
    cp[i] = c[i] / den;
    rp[i] = (r[i] - a[i] * rp[i - 1]) / den;
  }
  x.assign(m, real(0.0));
  x[m - 1] = rp[m - 1];
  for (int i = m - 2; i >= 0; --i) x[i] = rp[i] - cp[i] * x[i + 1];
}

// IG4 on a periodic line of n values: fp points at f_0 with f_{-2} .. f_{n+1} readable.
// The cyclic system (corners alpha) is solved with the Sherman-Morrison formula: with
// gamma = -b_0, A = T + u v^T, u = (gamma, 0.., alpha), v = (1, 0.., alpha/gamma); solve
// T y = r and T z = u, then x = y - (v.y)/(1 + v.z) z.
static void ig4_line_cyclic(const real* fp, int n, std::vector<real>& g) {
  const double al = kIG4Alpha;
  std::vector<real> a(n, real(al)), b(n, real(1.0)), c(n, real(al)), r(n), u(n, real(0.0));
  for (int i = 0; i < n; ++i) r[i] = ig4_rhs(fp, i);
  const real gamma = -b[0];
  b[0] = b[0] - gamma;
  b[n - 1] = b[n - 1] - al * al / gamma;
  a[0] = 0.0;
  c[n - 1] = 0.0;
  u[0] = gamma;
  u[n - 1] = al;
  std::vector<real> y, z;
  thomas(a, b, c, r, y);
  thomas(a, b, c, u, z);
  const real fac = (y[0] + al / gamma * y[n - 1]) / (1.0 + z[0] + al / gamma * z[n - 1]);
  g.assign(n, real(0.0));
  for (int i = 0; i < n; ++i) g[i] = y[i] - fac * z[i];
}

// IG4 on an open line of m >= 7 values: the three end points at each side take explicit
// rows (App. C, with the second cell's printed stencil shifted back by one index): second-order one-sided at the end
// point, fourth-order biased next to it, fourth-order central (Eq. 4thorder-grads) third;
// IG4 rows in between.
static void ig4_line_open(const real* f, int m, std::vector<real>& g) {
  const double al = kIG4Alpha;
  std::vector<real> a(m, real(al)), b(m, real(1.0)), c(m, real(al)), r(m, real(0.0));
  for (int t = 0; t < 3; ++t) {
    a[t] = c[t] = a[m - 1 - t] = c[m - 1 - t] = 0.0;
  }
  r[0] = -1.5 * f[0] + 2.0 * f[1] - 0.5 * f[2];
  r[1] = -0.25 * f[0] - (5.0 / 6.0) * f[1] + 1.5 * f[2] - 0.5 * f[3] + f[4] / 12.0;
  r[2] = (2.0 / 3.0) * (f[3] - f[1]) - (f[4] - f[0]) / 12.0;
  const int e = m - 1;
  r[e] = 1.5 * f[e] - 2.0 * f[e - 1] + 0.5 * f[e - 2];
  r[e - 1] = 0.25 * f[e] + (5.0 / 6.0) * f[e - 1] - 1.5 * f[e - 2] + 0.5 * f[e - 3] - f[e - 4] / 12.0;
  r[e - 2] = (2.0 / 3.0) * (f[e - 1] - f[e - 3]) - (f[e] - f[e - 4]) / 12.0;
  for (int i = 3; i < m - 3; ++i) r[i] = ig4_rhs(f, i);
  thomas(a, b, c, r, g);
}

// IG4 first derivatives of a padded field along d (output box: f's box shrunk by 3 along d,
// like op_e6).  Periodic axis: the cyclic system over the n cells, extended periodically;
// open axis: the whole padded line with explicit end rows.
static Field op_ig4(const Field& f, int d, bool periodic, int n) {
  Field o(f.b.grow(d, -3, -3));
  Box lines = o.b;
  lines.lo[d] = 0;
  lines.hi[d] = 1;
  const int flo = f.b.lo[d], fhi = f.b.hi[d];
  FOR_BOX(lines) {
    int c[3] = {i, j, k};
    std::vector<real> line(fhi - flo), g;
    for (int m = flo; m < fhi; ++m) {
      c[d] = m;
      line[m - flo] = f.at(c[0], c[1], c[2]);
    }
    if (periodic) {
      ig4_line_cyclic(line.data() - flo, n, g);
      for (int m = o.b.lo[d]; m < o.b.hi[d]; ++m) {
        c[d] = m;
        o.at(c[0], c[1], c[2]) = g[((m % n) + n) % n];
      }
    } else {
      ig4_line_open(line.data(), fhi - flo, g);
      for (int m = o.b.lo[d]; m < o.b.hi[d]; ++m) {
        c[d] = m;
        o.at(c[0], c[1], c[2]) = g[m - flo];
      }
    }
  }
  return o;
}

// Sec. 5.1 step 1, second derivative shared by MEG6 and MIG4:
// f''_i = 2 (f_{i+1} - 2 f_i + f_{i-1}) - 0.5 (f'_{i+1} - f'_{i-1})
static Field op_second(const Field& f, const Field& f1, int d) {
  Field o(box_and(f1.b.grow(d, -1, -1), f.b.grow(d, -1, -1)));
  FOR_BOX(o.b) {
    o.at(i, j, k) = 2.0 * (f.sh(i, j, k, d, 1) - 2.0 * f.at(i, j, k) + f.sh(i, j, k, d, -1)) -
                    0.5 * (f1.sh(i, j, k, d, 1) - f1.sh(i, j, k, d, -1));
  }
  return o;
}

// Eq. (FP-interp) / (interp-formulae): central interface value at i+1/2 as the
// average of the van Leer left and right states of Eq. (vanleer-poly).
// Output index i holds the interface i+1/2.
static Field op_face(const Field& f, const Field& f1, const Field& f2, int d) {
  Box ob = f2.b;
  ob.hi[d] -= 1;
  Field o(ob);
  FOR_BOX(o.b) {
    real left = f.at(i, j, k) + 0.5 * f1.at(i, j, k) + f2.at(i, j, k) / 12.0;
    real right = f.sh(i, j, k, d, 1) - 0.5 * f1.sh(i, j, k, d, 1) + f2.sh(i, j, k, d, 1) / 12.0;
    o.at(i, j, k) = 0.5 * (left + right);
  }
  return o;
}

// Eq. (FP-interp2) and the flux difference of Sec. 3: (f_{i+1/2} - f_{i-1/2}) / dxi, dxi = 1.
static Field op_delta(const Field& fc, int d) {
  Box ob = fc.b;
  ob.lo[d] += 1;
  Field o(ob);
  FOR_BOX(o.b) { o.at(i, j, k) = fc.at(i, j, k) - fc.sh(i, j, k, d, -1); }
  return o;
}

// Interpolation of a cell field to interfaces, Sec. 7 step 3 (scheme 0: E6
// gradients; scheme 1: the E4 gradients of App. D).
static Field op_interp(const Field& f, int d, int scheme) {
  Field f1 = scheme ? op_e4(f, d) : op_e6(f, d);
  Field f2 = op_second(f, f1, d);
  return op_face(f, f1, f2, d);
}

// Sec. 7 step 2: consistent metric derivative D = delta o interp (MEG6).
static Field op_D(const Field& f, int d) { return op_delta(op_interp(f, d, 0), d); }

// Sec. 7 steps 2-3 for MIG4: the same interpolation and derivative, with x' from the IG4
// system (Eq. IG4_grads) solved over the field's whole line along d with the explicit end
// rows.  On a periodic axis the geometry line is the unwrapped line extended kExtIG4 cells
// beyond each side, so this is IG4 on the unbounded line: the inverse of the (alpha, 1, alpha)
// operator decays by |r| = 0.4226 per cell, and the end rows reach the cells that are kept
// below 1e-20 of their own size.
static Field op_interp_ig4(const Field& f, int d) {
  Field f1 = op_ig4(f, d, false, 0);
  Field f2 = op_second(f, f1, d);
  return op_face(f, f1, f2, d);
}

// ---------------------------------------------------------------------------
// App. C: an axis bounded by walls on both sides (no ghost nodes).
// The field's box along d is the n cells [lo, hi); the first and last three
// cells take one-sided derivatives, the interfaces next to the walls one-sided
// states, so that D = delta o interp is defined on every cell and is the same
// operator in every line (the metric identities of Sec. 7 still hold).
// ---------------------------------------------------------------------------
// first derivative on the whole box
static Field op_e6_c(const Field& f, int d) {
  Field o(f.b);
  const int lo = f.b.lo[d], hi = f.b.hi[d];
  FOR_BOX(o.b) {
    int c[3] = {i, j, k};
    const int m = c[d];
    auto F = [&](int s) { return f.sh(i, j, k, d, s); };
    real v;
    if (m == lo) v = -1.5 * F(0) + 2.0 * F(1) - 0.5 * F(2);                       // 2nd order one-sided
    else if (m == hi - 1) v = 1.5 * F(0) - 2.0 * F(-1) + 0.5 * F(-2);
    else if (m == lo + 1)                                                           // 4th order biased (printed stencil shifted back by one index)
      v = -0.25 * F(-1) - (5.0 / 6.0) * F(0) + 1.5 * F(1) - 0.5 * F(2) + F(3) / 12.0;
    else if (m == hi - 2) v = 0.25 * F(1) + (5.0 / 6.0) * F(0) - 1.5 * F(-1) + 0.5 * F(-2) - F(-3) / 12.0;
    else if (m == lo + 2 || m == hi - 3)                                            // 4th order central
      v = (2.0 / 3.0) * (F(1) - F(-1)) - (F(2) - F(-2)) / 12.0;
    else
      v = (3.0 / 4.0) * (F(1) - F(-1)) - (3.0 / 20.0) * (F(2) - F(-2)) + (1.0 / 60.0) * (F(3) - F(-3));
    o.at(i, j, k) = v;
  }
  return o;
}

// second derivative on the whole box: one-sided derivatives of f' in the two end cells,
// the interior formula of Sec. 5.1 elsewhere (the third cell takes the interior formula: the printed one is garbled)
static Field op_second_c(const Field& f, const Field& f1, int d) {
  Field o(f.b);
  const int lo = f.b.lo[d], hi = f.b.hi[d];
  FOR_BOX(o.b) {
    int c[3] = {i, j, k};
    const int m = c[d];
    auto G = [&](int s) { return f1.sh(i, j, k, d, s); };
    real v;
    if (m == lo) v = -1.5 * G(0) + 2.0 * G(1) - 0.5 * G(2);
    else if (m == hi - 1) v = 1.5 * G(0) - 2.0 * G(-1) + 0.5 * G(-2);
    else if (m == lo + 1) v = -0.25 * G(-1) - (5.0 / 6.0) * G(0) + 1.5 * G(1) - 0.5 * G(2) + G(3) / 12.0;
    else if (m == hi - 2) v = 0.25 * G(1) + (5.0 / 6.0) * G(0) - 1.5 * G(-1) + 0.5 * G(-2) - G(-3) / 12.0;
    else
      v = 2.0 * (f.sh(i, j, k, d, 1) - 2.0 * f.at(i, j, k) + f.sh(i, j, k, d, -1)) - 0.5 * (G(1) - G(-1));
    o.at(i, j, k) = v;
  }
  return o;
}

// interface values i+1/2 for i = lo-1 .. hi-1 (the two walls included): the wall interfaces take
// the boundary cell's own state on that side; the interfaces between the first two and the last
// two cells take the state of the inner cell only (App. C); the others the mean of both states
static Field op_face_c(const Field& f, const Field& f1, const Field& f2, int d) {
  Box ob = f.b;
  const int lo = f.b.lo[d], hi = f.b.hi[d];
  ob.lo[d] = lo - 1;
  Field o(ob);
  FOR_BOX(o.b) {
    int c[3] = {i, j, k};
    const int m = c[d];
    auto left = [&]() {  // state of cell m at its + face
      return f.at(i, j, k) + 0.5 * f1.at(i, j, k) + f2.at(i, j, k) / 12.0;
    };
    auto right = [&]() {  // state of cell m+1 at its - face
      return f.sh(i, j, k, d, 1) - 0.5 * f1.sh(i, j, k, d, 1) + f2.sh(i, j, k, d, 1) / 12.0;
    };
    real v;
    if (m == lo - 1) v = right();
    else if (m == hi - 1) v = left();
    else if (m == lo) v = right();
    else if (m == hi - 2) v = left();
    else v = 0.5 * (left() + right());
    o.at(i, j, k) = v;
  }
  return o;
}

static Field op_interp_c(const Field& f, int d) {
  Field f1 = op_e6_c(f, d);
  Field f2 = op_second_c(f, f1, d);
  return op_face_c(f, f1, f2, d);
}

static Field f_mul(const Field& a, const Field& b) {
  Field o(box_and(a.b, b.b));
  FOR_BOX(o.b) { o.at(i, j, k) = a.at(i, j, k) * b.at(i, j, k); }
  return o;
}
static Field f_sub(const Field& a, const Field& b) {
  Field o(box_and(a.b, b.b));
  FOR_BOX(o.b) { o.at(i, j, k) = a.at(i, j, k) - b.at(i, j, k); }
  return o;
}
static Field f_crop(const Field& a, const Box& b) {
  Field o(b);
  FOR_BOX(o.b) { o.at(i, j, k) = a.at(i, j, k); }
  return o;
}

// ---------------------------------------------------------------------------
// Eigenvectors (App. A), HLLC (Sec. 5.1.1), MP limiter (App. E)
// ---------------------------------------------------------------------------

// Structural nonzeros of the App. A matrices; products skip the structural zeros.
static const int NZ_R3[5][5] = {{1, 1, 1, 1, 1}, {1, 0, 1, 1, 1}, {1, 1, 1, 0, 1}, {1, 1, 0, 1, 1}, {1, 0, 0, 0, 1}};
static const int NZ_L3[5][5] = {{0, 1, 1, 1, 1}, {1, 0, 1, 1, 1}, {1, 1, 1, 0, 1}, {1, 1, 0, 1, 1}, {0, 1, 1, 1, 1}};
static const int NZ_R2[4][4] = {{1, 1, 0, 1}, {1, 0, 1, 1}, {1, 0, 1, 1}, {1, 0, 0, 1}};
static const int NZ_L2[4][4] = {{0, 1, 1, 1}, {1, 0, 0, 1}, {0, 1, 1, 0}, {0, 1, 1, 1}};

static int nz_of(int nd, int left, int r, int c) {
  if (nd == 3) return left ? NZ_L3[r][c] : NZ_R3[r][c];
  return left ? NZ_L2[r][c] : NZ_R2[r][c];
}

// App. A: right (R) and left (R^{-1}) eigenvectors of B_xi in primitive
// variables P = [rho, u, v, w, p], with the normalised metric n~ = n^/|n^|
// and the face density and speed of sound.  2D: the restriction to
// P = [rho, u, v, p] (the entropy row is n~x row1 - n~y row3).
static void eigen(int nd, const real* nh, real rho, real p, real gamma, real R[5][5], real L[5][5]) {
  real nn2 = 0.0;
  for (int a = 0; a < nd; ++a) nn2 = nn2 + nh[a] * nh[a];
  real nn = Sqrt(nn2);
  real n0 = nh[0] / nn, n1 = nh[1] / nn, n2 = (nd == 3) ? nh[2] / nn : real(0.0);
  real a = Sqrt(gamma * p / rho);
  real a2 = a * a;
  real ra = rho * a;
  for (int r = 0; r < 5; ++r)
    for (int c = 0; c < 5; ++c) R[r][c] = L[r][c] = 0.0;
  if (nd == 3) {
    R[0][0] = 1.0 / (2.0 * a2); R[0][1] = n0 / a2;  R[0][2] = n2 / a2; R[0][3] = -n1 / a2; R[0][4] = 1.0 / (2.0 * a2);
    R[1][0] = -n0 / (2.0 * ra); R[1][2] = -n1;      R[1][3] = -n2;     R[1][4] = n0 / (2.0 * ra);
    R[2][0] = -n1 / (2.0 * ra); R[2][1] = -n2;      R[2][2] = n0;      R[2][4] = n1 / (2.0 * ra);
    R[3][0] = -n2 / (2.0 * ra); R[3][1] = n1;       R[3][3] = n0;      R[3][4] = n2 / (2.0 * ra);
    R[4][0] = 0.5;              R[4][4] = 0.5;

    L[0][1] = -n0 * ra; L[0][2] = -n1 * ra; L[0][3] = -n2 * ra; L[0][4] = 1.0;
    L[1][0] = n0 * a2;  L[1][2] = -n2;      L[1][3] = n1;       L[1][4] = -n0;
    L[2][0] = n2 * a2;  L[2][1] = -n1;      L[2][2] = n0;       L[2][4] = -n2;
    L[3][0] = -n1 * a2; L[3][1] = -n2;      L[3][3] = n0;       L[3][4] = n1;
    L[4][1] = n0 * ra;  L[4][2] = n1 * ra;  L[4][3] = n2 * ra;  L[4][4] = 1.0;
  } else {
    R[0][0] = 1.0 / (2.0 * a2); R[0][1] = 1.0 / a2; R[0][3] = 1.0 / (2.0 * a2);
    R[1][0] = -n0 / (2.0 * ra); R[1][2] = -n1;      R[1][3] = n0 / (2.0 * ra);
    R[2][0] = -n1 / (2.0 * ra); R[2][2] = n0;       R[2][3] = n1 / (2.0 * ra);
    R[3][0] = 0.5;              R[3][3] = 0.5;

    L[0][1] = -n0 * ra; L[0][2] = -n1 * ra; L[0][3] = 1.0;
    L[1][0] = a2;       L[1][3] = -1.0;
    L[2][1] = -n1;      L[2][2] = n0;
    L[3][1] = n0 * ra;  L[3][2] = n1 * ra;  L[3][3] = 1.0;
  }
}

static void matvec(int nd, int left, const real M[5][5], const real* x, real* y) {
  const int nv = nd + 2;
  for (int r = 0; r < nv; ++r) {
    bool first = true;
    real acc = 0.0;
    for (int c = 0; c < nv; ++c) {
      if (!nz_of(nd, left, r, c)) continue;
      if (first) { acc = M[r][c] * x[c]; first = false; }
      else acc = acc + M[r][c] * x[c];
    }
    y[r] = acc;
  }
}

// Sec. 5.1.1: HLLC in curvilinear coordinates with grid motion.
// P = [rho, u_1..u_nd, p]; nh = face hat metric (xi^_x, xi^_y, xi^_z); nt = xi^_t.
static void hllc(int nd, const real* PL, const real* PR, const real* nh, real nt, real gamma, real* F) {
  const int nv = nd + 2;
  real nn2 = 0.0;
  for (int a = 0; a < nd; ++a) nn2 = nn2 + nh[a] * nh[a];
  real nn = Sqrt(nn2);

  real rho[2], u[2][3], p[2], En[2], U[2], c[2];
  const real* Ps[2] = {PL, PR};
  for (int s = 0; s < 2; ++s) {
    rho[s] = Ps[s][0];
    real q2 = 0.0;
    U[s] = nt;
    for (int a = 0; a < nd; ++a) {
      u[s][a] = Ps[s][1 + a];
      q2 = q2 + u[s][a] * u[s][a];
      U[s] = U[s] + nh[a] * u[s][a];  // contravariant velocity, Sec. 2
    }
    p[s] = Ps[s][nv - 1];
    En[s] = p[s] / (gamma - 1.0) + 0.5 * rho[s] * q2;  // energy per unit volume, Sec. 2
    c[s] = Sqrt(gamma * p[s] / rho[s]);
  }
  // wave speeds
  real SL = Min(U[0] - c[0] * nn, U[1] - c[1] * nn);
  real SR = Max(U[0] + c[0] * nn, U[1] + c[1] * nn);
  real Ss = (rho[1] * U[1] * (SR - U[1]) - rho[0] * U[0] * (SL - U[0]) + (p[0] - p[1]) * nn2) /
            (rho[1] * (SR - U[1]) - rho[0] * (SL - U[0]));

  // physical flux of side s (Eq. inv_fluxes)
  auto phys = [&](int s, real* Fo) {
    Fo[0] = rho[s] * U[s];
    for (int a = 0; a < nd; ++a) Fo[1 + a] = rho[s] * u[s][a] * U[s] + nh[a] * p[s];
    Fo[nv - 1] = (En[s] + p[s]) * U[s] - nt * p[s];
  };
  // star-region flux F*K = F^K + S^K (Q*K - Q^K)
  auto star = [&](int s, real S, real* Fo) {
    real Fk[5];
    phys(s, Fk);
    real fac = rho[s] * ((S - U[s]) / (S - Ss));
    real Qs[5], Qk[5];
    Qs[0] = fac * 1.0;
    for (int a = 0; a < nd; ++a) {
      real num = nh[a] * (Ss - nt);
      for (int b = 0; b < nd; ++b) {
        real coef;
        if (b == a) {
          coef = 0.0;
          for (int e = 0; e < nd; ++e)
            if (e != a) coef = coef + nh[e] * nh[e];
        } else {
          coef = -(nh[b] * nh[a]);
        }
        num = num + coef * u[s][b];
      }
      Qs[1 + a] = fac * (num / nn2);
    }
    Qs[nv - 1] = fac * (En[s] / rho[s] + (Ss - U[s]) * ((Ss - nt) / nn2 + p[s] / (rho[s] * (S - U[s]))));
    Qk[0] = rho[s];
    for (int a = 0; a < nd; ++a) Qk[1 + a] = rho[s] * u[s][a];
    Qk[nv - 1] = En[s];
    for (int m = 0; m < nv; ++m) Fo[m] = Fk[m] + S * (Qs[m] - Qk[m]);
  };
  if (SL >= 0.0) {
    phys(0, F);
  } else if (Ss >= 0.0) {
    star(0, SL, F);
  } else if (SR > 0.0) {
    star(1, SR, F);
  } else {
    phys(1, F);
  }
}

// App. E, improved MP limiter, written for the left-biased state of the base
// cell: w_up is the upwind neighbour (i-1), w_base the base cell (i), w_down the
// downwind neighbour (i+1); d_* are the curvatures d of those cells.  The right
// state at i+1/2 uses the mirror image (up = i+2, base = i+1, down = i).
static real mp_limit(real wf, real w_up, real w_base, real w_down, real d_up, real d_base, real d_down, real alpha,
                     real beta, real eps) {
  real wmp = w_base + minmod(w_down - w_base, beta * (w_base - w_up));
  if ((wf - w_base) * (wf - wmp) <= eps) return wf;
  real dm_down = minmod(d_base, d_down);  // d^M_{i+1/2}
  real dm_up = minmod(d_up, d_base);      // d^M_{i-1/2}
  real wmd = 0.5 * (w_base + w_down) - 0.5 * dm_down;
  real wul = w_base + alpha * (w_base - w_up);
  real wlc = 0.5 * (3.0 * w_base - w_up) + (4.0 / 3.0) * dm_up;
  real wmin = Max(Min3(w_base, w_down, wmd), Min3(w_base, wul, wlc));
  real wmax = Min(Max3(w_base, w_down, wmd), Max3(w_base, wul, wlc));
  return wf + minmod(wmin - wf, wmax - wf);
}

// ---------------------------------------------------------------------------
// Solver state
// ---------------------------------------------------------------------------
struct Geom {
  Field mh[3][3];     // cell hat metrics m^[e][a] = (d xi_e / d x_a) / J
  Field det;          // cell 1/J (determinant, Eq. Jac-matrix)
  Field mt[3];        // cell hat time metrics xi^_t, eta^_t, zeta^_t
  Field fh[3][3];     // face hat metrics of direction d: fh[d][a]
  Field fu[3][3][3];  // face unhatted metrics fu[d][e][a] (viscous chain rule)
  Field ft[3];        // face hat time metric of direction d
  Field gcl;          // (1/J)_t at interior cells (Eq. Jacb2)
  bool moving = false;
};

struct orc_solver {
  orc_params p;
  int nd = 3, nv = 5;
  bool viscous = false;
  bool closed[3] = {false, false, false};  // wall-bounded axis without ghost nodes (App. C)
  Box inner, pad, ext, cellgeo;
  Geom g;
  std::vector<double> inflow;  // [nv][nk][nj] primitives for an x-low inflow side
  std::vector<double> sigma, qamb;

  int build_geometry(const Field* xc, const Field* vc);
  int centroids_from_nodes(const double* nodes, const double* vel, Field* xc, Field* vc);
  void fill_ghosts(Field* P) const;
  int rhs(const double* q, double* Lout, double* resout, int fdir, double* gout, double* primout);
  void face_flux(int d, int i, int j, int k, const Field* P, const Field (*P1)[5], const Field (*P2)[5],
                 const Field& T, const Field* T1, real* G) const;
  real viscosity(real T) const;
};

static Box make_box(int nd, const int* n, int pad) {
  Box b;
  for (int d = 0; d < 3; ++d) {
    if (d < nd) { b.lo[d] = -pad; b.hi[d] = n[d] + pad; }
    else { b.lo[d] = 0; b.hi[d] = 1; }
  }
  return b;
}

// Sec. 3: the solution lives at the centroid of the cell's vertices.  Periodic
// axes are extended with unwrapped images (node n = node 0 + period vector);
// non-periodic axes use the ghost node layers supplied by the caller.
int orc_solver::centroids_from_nodes(const double* nodes, const double* vel, Field* xc, Field* vc) {
  const int G = p.ghost_nodes;
  int Nn[3], off[3];
  for (int d = 0; d < 3; ++d) {
    if (d >= nd) { Nn[d] = 1; off[d] = 0; continue; }
    if (p.periodic[d]) { Nn[d] = p.n[d] + 1; off[d] = 0; }
    else { Nn[d] = p.n[d] + 1 + 2 * G; off[d] = G; }
  }
  auto nid = [&](int si, int sj, int sk) { return ((size_t)sk * Nn[1] + sj) * Nn[0] + si; };
  const size_t NN = (size_t)Nn[0] * Nn[1] * Nn[2];
  // period vectors
  double per[3][3] = {{0}};
  double scale = 0.0;
  for (size_t m = 0; m < (size_t)nd * NN; ++m) scale = std::fmax(scale, std::fabs(nodes[m]));
  for (int d = 0; d < nd; ++d) {
    if (!p.periodic[d]) continue;
    int s0[3] = {off[0], off[1], off[2]};
    int s1[3] = {off[0], off[1], off[2]};
    s1[d] = p.n[d];
    for (int a = 0; a < nd; ++a) per[d][a] = nodes[a * NN + nid(s1[0], s1[1], s1[2])] - nodes[a * NN + nid(s0[0], s0[1], s0[2])];
    // closure check over every node of the closing face
    for (int sk = 0; sk < Nn[2]; ++sk)
      for (int sj = 0; sj < Nn[1]; ++sj)
        for (int si = 0; si < Nn[0]; ++si) {
          int s[3] = {si, sj, sk};
          if (s[d] != 0) continue;
          int t[3] = {si, sj, sk};
          t[d] = p.n[d];
          for (int a = 0; a < nd; ++a) {
            double diff = nodes[a * NN + nid(t[0], t[1], t[2])] - nodes[a * NN + nid(s[0], s[1], s[2])];
            if (std::fabs(diff - per[d][a]) > 1e-12 * (scale + 1.0))
              return fail("periodic axis is not closed by a constant period vector");
          }
        }
  }
  // node position (axis a) at extended node index m (m may lie outside [0, n])
  auto node_at = [&](const double* arr, const int* m, int a, bool shift) -> double {
    int s[3];
    double add = 0.0;
    for (int d = 0; d < 3; ++d) {
      if (d >= nd) { s[d] = 0; continue; }
      if (p.periodic[d]) {
        int n = p.n[d];
        int base = ((m[d] % n) + n) % n;
        int wraps = (m[d] - base) / n;
        s[d] = base;
        if (shift) add += wraps * per[d][a];
      } else {
        s[d] = m[d] + off[d];
      }
    }
    return arr[a * NN + nid(s[0], s[1], s[2])] + add;
  };
  for (int a = 0; a < nd; ++a) {
    xc[a] = Field(ext);
    if (vel) vc[a] = Field(ext);
  }
  const int nc = (nd == 3) ? 8 : 4;
  for (int a = 0; a < nd; ++a) {
    FOR_BOX(ext) {
      real sx = 0.0, sv = 0.0;
      for (int ck = 0; ck < (nd == 3 ? 2 : 1); ++ck)
        for (int cj = 0; cj < 2; ++cj)
          for (int ci = 0; ci < 2; ++ci) {
            int m[3] = {i + ci, j + cj, k + ck};
            sx = sx + node_at(nodes, m, a, true);
            if (vel) sv = sv + node_at(vel, m, a, false);
          }
      xc[a].at(i, j, k) = sx / (double)nc;
      if (vel) vc[a].at(i, j, k) = sv / (double)nc;
    }
  }
  return 0;
}

// Sec. 4 and Sec. 7: conservative metrics, Jacobian, time metrics, face
// interpolation and the GCL term.  xc/vc: centroids (velocities) on ext.
int orc_solver::build_geometry(const Field* xc, const Field* vc) {
  ORC_PHASE(PH_GEOM);
  const int sch = p.metric_scheme;
  Field xd[3][3];  // xd[a][d] = d x_a / d xi_d
  // Sec. 7 operators built from the scheme's own gradients (step 2): E6 for MEG6, IG4 for MIG4;
  // App. C on wall-bounded axes; the E4 operators of App. D for the non-conservative control
  const bool ig4 = sch == 0 && p.gradient_scheme == 1;
  auto Iop = [&](const Field& f, int d) {
    if (closed[d]) return op_interp_c(f, d);
    return ig4 ? op_interp_ig4(f, d) : op_interp(f, d, sch);
  };
  auto Dop = [&](const Field& f, int d) { return op_delta(Iop(f, d), d); };
  for (int a = 0; a < nd; ++a)
    for (int d = 0; d < nd; ++d) xd[a][d] = sch == 0 ? Dop(xc[a], d) : op_e4(xc[a], d);

  Field mh[3][3];
  Field det;
  if (nd == 3) {
    for (int e = 0; e < 3; ++e) {
      int f = (e + 1) % 3, gg = (e + 2) % 3;
      for (int a = 0; a < 3; ++a) {
        int b = (a + 1) % 3, c = (a + 2) % 3;
        if (sch == 0) {
          // Eq. (GCL_metrics): e.g. xi^_x = (y_eta z)_zeta - (y_zeta z)_eta
          mh[e][a] = f_sub(Dop(f_mul(xd[b][f], xc[c]), gg), Dop(f_mul(xd[b][gg], xc[c]), f));
        } else {
          // App. D: e.g. xi^_x = y_eta z_zeta - y_zeta z_eta (the cyclic form; the printed zeta^_y swaps the indices)
          mh[e][a] = f_sub(f_mul(xd[b][f], xd[c][gg]), f_mul(xd[b][gg], xd[c][f]));
        }
      }
    }
    Box db = xd[0][0].b;
    for (int a = 0; a < 3; ++a)
      for (int d = 0; d < 3; ++d) db = box_and(db, xd[a][d].b);
    det = Field(db);
    FOR_BOX(db) {
      real xx = xd[0][0].at(i, j, k), yx = xd[1][0].at(i, j, k), zx = xd[2][0].at(i, j, k);
      real xe = xd[0][1].at(i, j, k), ye = xd[1][1].at(i, j, k), ze = xd[2][1].at(i, j, k);
      real xz = xd[0][2].at(i, j, k), yz = xd[1][2].at(i, j, k), zz = xd[2][2].at(i, j, k);
      // Eq. (Jac-matrix): rows (x_xi, y_xi, z_xi), (x_eta, ...), (x_zeta, ...)
      det.at(i, j, k) = xx * (ye * zz - ze * yz) - yx * (xe * zz - ze * xz) + zx * (xe * yz - ye * xz);
    }
  } else {
    // 2D: the 3D formulas with z = zeta
    Field neg_xe(xd[0][1].b), neg_yx(xd[1][0].b);
    FOR_BOX(neg_xe.b) { neg_xe.at(i, j, k) = -xd[0][1].at(i, j, k); }
    FOR_BOX(neg_yx.b) { neg_yx.at(i, j, k) = -xd[1][0].at(i, j, k); }
    mh[0][0] = xd[1][1];  // xi^_x  =  y_eta
    mh[0][1] = neg_xe;    // xi^_y  = -x_eta
    mh[1][0] = neg_yx;    // eta^_x = -y_xi
    mh[1][1] = xd[0][0];  // eta^_y =  x_xi
    Box db = box_and(box_and(xd[0][0].b, xd[0][1].b), box_and(xd[1][0].b, xd[1][1].b));
    det = Field(db);
    FOR_BOX(db) {
      det.at(i, j, k) = xd[0][0].at(i, j, k) * xd[1][1].at(i, j, k) - xd[0][1].at(i, j, k) * xd[1][0].at(i, j, k);
    }
  }
  for (int e = 0; e < nd; ++e)
    for (int a = 0; a < nd; ++a) {
      if (!mh[e][a].b.contains(cellgeo)) return fail("internal: metric box too small");
      g.mh[e][a] = f_crop(mh[e][a], cellgeo);
    }
  if (!det.b.contains(cellgeo)) return fail("internal: det box too small");
  g.det = f_crop(det, cellgeo);
  {
    double dmin = std::numeric_limits<double>::infinity();
    for (size_t m = 0; m < g.det.v.size(); ++m) dmin = std::fmin(dmin, Dbl(g.det.v[m]));
    if (!(dmin > 0.0)) return fail("non-positive cell volume 1/J");
  }

  // Sec. 4: xi_t = -(x_t xi_x + y_t xi_y + z_t xi_z); in hat form with the cell grid velocity
  g.moving = (vc != nullptr);
  if (g.moving) {
    for (int e = 0; e < nd; ++e) {
      g.mt[e] = Field(cellgeo);
      FOR_BOX(cellgeo) {
        real s = 0.0;
        for (int a = 0; a < nd; ++a) s = s + vc[a].at(i, j, k) * g.mh[e][a].at(i, j, k);
        g.mt[e].at(i, j, k) = -s;
      }
    }
  }

  // Sec. 7 step 3: interpolate whole products (xi_x/J) to interfaces
  for (int d = 0; d < nd; ++d) {
    Box fb = inner;
    fb.lo[d] = -1;
    fb.hi[d] = p.n[d];
    for (int a = 0; a < nd; ++a) g.fh[d][a] = f_crop(Iop(g.mh[d][a], d), fb);
    if (viscous) {
      for (int e = 0; e < nd; ++e)
        for (int a = 0; a < nd; ++a) {
          Field m(cellgeo);  // unhatted cell metric xi_x = (xi_x/J) * J
          FOR_BOX(cellgeo) { m.at(i, j, k) = g.mh[e][a].at(i, j, k) / g.det.at(i, j, k); }
          g.fu[d][e][a] = f_crop(Iop(m, d), fb);
        }
    }
    if (g.moving) g.ft[d] = f_crop(Iop(g.mt[d], d), fb);
  }
  // Eq. (Jacb2) on the face values, the same difference as the flux divergence
  g.gcl = Field(inner);
  if (g.moving) {
    FOR_BOX(inner) {
      real s = 0.0;
      for (int d = 0; d < nd; ++d) s = s + (g.ft[d].at(i, j, k) - g.ft[d].sh(i, j, k, d, -1));
      g.gcl.at(i, j, k) = -s;
    }
  }
  ORC_PHASE(PH_MISC);
  return 0;
}

real orc_solver::viscosity(real T) const {
  real mu_ref = 1.0 / p.reynolds;
  if (!(p.sutherland_s > 0.0)) return mu_ref;
  // Sutherland's law (Sec. 2), read as: mu = mu_ref th^{3/2} (1 + S)/(th + S), th = T/T_ref
  real th = T / p.t_ref;
  return mu_ref * (th * Sqrt(th)) * ((1.0 + p.sutherland_s) / (th + p.sutherland_s));
}

// Ghost layers of the primitive variables (Sec. 5): periodic copy, zero
// gradient, or Dirichlet inflow.  Axis by axis, so edges and corners are filled.
void orc_solver::fill_ghosts(Field* P) const {
  for (int d = 0; d < nd; ++d) {
    Box S = inner;
    for (int e = 0; e < d; ++e) { S.lo[e] = pad.lo[e]; S.hi[e] = pad.hi[e]; }
    S.lo[d] = 0;
    S.hi[d] = 1;  // loop over the cross-section only
    const int n = p.n[d];
    for (int c = 0; c < nv; ++c) {
      Field& f = P[c];
      FOR_BOX(S) {
        int lo[3] = {i, j, k}, hi[3] = {i, j, k}, src[3] = {i, j, k};
        for (int gl = 1; gl <= H; ++gl) {
          lo[d] = -gl;
          hi[d] = n - 1 + gl;
          if (p.periodic[d]) {
            src[d] = n - gl;
            f.at(lo[0], lo[1], lo[2]) = f.at(src[0], src[1], src[2]);
            src[d] = gl - 1;
            f.at(hi[0], hi[1], hi[2]) = f.at(src[0], src[1], src[2]);
          } else {
            if (p.bc[d][0] == ORC_BC_INFLOW) {
              f.at(lo[0], lo[1], lo[2]) = inflow[((size_t)c * p.n[2] + k) * p.n[1] + j];
            } else {
              src[d] = 0;
              f.at(lo[0], lo[1], lo[2]) = f.at(src[0], src[1], src[2]);
            }
            src[d] = n - 1;
            f.at(hi[0], hi[1], hi[2]) = f.at(src[0], src[1], src[2]);
          }
        }
      }
    }
    // slip walls: ghost layer g mirrors cell g - 1 (n - g on the high side) --
    // density and pressure as they are, the velocity reflected about the unit normal of the
    // wall face, taken at the cross-section (coordinates of earlier axes clamped to the cells)
    for (int side = 0; side < 2; ++side) {
      if (p.periodic[d] || p.bc[d][side] != ORC_BC_WALL) continue;
      FOR_BOX(S) {
        int fc[3] = {i, j, k};
        for (int e = 0; e < nd; ++e)
          if (e != d) fc[e] = fc[e] < 0 ? 0 : (fc[e] >= p.n[e] ? p.n[e] - 1 : fc[e]);
        fc[d] = side == 0 ? -1 : n - 1;  // the wall interface
        real nh[3] = {0.0, 0.0, 0.0}, nn = 0.0;
        for (int a = 0; a < nd; ++a) {
          nh[a] = g.fh[d][a].at(fc[0], fc[1], fc[2]);
          nn = nn + nh[a] * nh[a];
        }
        const real inv = 1.0 / Sqrt(nn);
        for (int a = 0; a < nd; ++a) nh[a] = nh[a] * inv;
        for (int gl = 1; gl <= H; ++gl) {
          int gc[3] = {i, j, k}, sc[3] = {i, j, k};
          gc[d] = side == 0 ? -gl : n - 1 + gl;
          sc[d] = side == 0 ? gl - 1 : n - gl;
          real un = 0.0;
          for (int a = 0; a < nd; ++a) un = un + P[1 + a].at(sc[0], sc[1], sc[2]) * nh[a];
          P[0].at(gc[0], gc[1], gc[2]) = P[0].at(sc[0], sc[1], sc[2]);
          P[nv - 1].at(gc[0], gc[1], gc[2]) = P[nv - 1].at(sc[0], sc[1], sc[2]);
          for (int a = 0; a < nd; ++a)
            P[1 + a].at(gc[0], gc[1], gc[2]) = P[1 + a].at(sc[0], sc[1], sc[2]) - 2.0 * un * nh[a];
        }
      }
    }
  }
}

// One interface i+1/2 (index (i,j,k) along d): Sec. 5.1 steps 2-6 and Sec. 5.2 steps 1-4.
void orc_solver::face_flux(int d, int i, int j, int k, const Field* P, const Field (*P1)[5], const Field (*P2)[5],
                           const Field& T, const Field* T1, real* G) const {
  const real gamma = p.gamma;
  int cc[4][3];
  for (int m = 0; m < 4; ++m) {
    cc[m][0] = i; cc[m][1] = j; cc[m][2] = k;
    cc[m][d] += m - 1;  // cells i-1, i, i+1, i+2
  }
#define CELL(m) cc[m][0], cc[m][1], cc[m][2]
  real nh[3] = {0.0, 0.0, 0.0};
  for (int a = 0; a < nd; ++a) nh[a] = g.fh[d][a].at(i, j, k);
  real nt = g.moving ? g.ft[d].at(i, j, k) : real(0.0);

  // Step 2: characteristic projection with the face eigenvectors (App. A).
  // Face state: arithmetic mean of rho and p of cells i and i+1.
  real rb = 0.5 * (P[0].at(CELL(1)) + P[0].at(CELL(2)));
  real pb = 0.5 * (P[nv - 1].at(CELL(1)) + P[nv - 1].at(CELL(2)));
  real R[5][5], Ri[5][5];
  eigen(nd, nh, rb, pb, gamma, R, Ri);
  real W[4][5], W2[4][5], W1[2][5], x[5];
  for (int m = 0; m < 4; ++m) {
    for (int c = 0; c < nv; ++c) x[c] = P[c].at(CELL(m));
    matvec(nd, 1, Ri, x, W[m]);
    for (int c = 0; c < nv; ++c) x[c] = P2[d][c].at(CELL(m));
    matvec(nd, 1, Ri, x, W2[m]);
  }
  for (int m = 0; m < 2; ++m) {
    for (int c = 0; c < nv; ++c) x[c] = P1[d][c].at(CELL(m + 1));
    matvec(nd, 1, Ri, x, W1[m]);
  }
  // Step 3: unlimited left/right states (Eq. legendre_polys); Step 4: App. E limiter
  // (d_i of App. E equals the projected second derivative W''_i with dx = 1).
  real WL[5], WR[5];
  for (int s = 0; s < nv; ++s) {
    real wl = W[1][s] + 0.5 * W1[0][s] + W2[1][s] / 12.0;
    real wr = W[2][s] - 0.5 * W1[1][s] + W2[2][s] / 12.0;
    WL[s] = mp_limit(wl, W[0][s], W[1][s], W[2][s], W2[0][s], W2[1][s], W2[2][s], p.mp_alpha, p.mp_beta, p.mp_eps);
    WR[s] = mp_limit(wr, W[3][s], W[2][s], W[1][s], W2[3][s], W2[2][s], W2[1][s], p.mp_alpha, p.mp_beta, p.mp_eps);
  }
  // Step 5: back to primitive variables
  real PL[5], PR[5];
  matvec(nd, 0, R, WL, PL);
  matvec(nd, 0, R, WR, PR);
  // Step 6: HLLC flux
  real F[5];
  hllc(nd, PL, PR, nh, nt, gamma, F);

  if (viscous) {
    // Sec. 5.2: alpha-damping, variables [u_1..u_nd, T]
    real gx[4][3];  // gx[v][a] = d phi_v / d x_a at the interface
    real phif[4];
    for (int v = 0; v <= nd; ++v) {
      auto val = [&](int m) -> real { return v < nd ? P[1 + v].at(CELL(m)) : T.at(CELL(m)); };
      auto grd = [&](int e, int m) -> real { return v < nd ? P1[e][1 + v].at(CELL(m)) : T1[e].at(CELL(m)); };
      real gc[3];
      // Eq. (AD-eqn2) with beta^D = 0
      real phiL = val(1) + 0.5 * grd(d, 1);
      real phiR = val(2) - 0.5 * grd(d, 2);
      for (int e = 0; e < nd; ++e) {
        if (e == d) gc[e] = 0.5 * (grd(e, 1) + grd(e, 2)) + (p.alpha_damping / 2.0) * (phiR - phiL);  // Eq. (AD-eqn1)
        else gc[e] = 0.5 * (grd(e, 1) + grd(e, 2));  // tangential: mean of the cell gradients
      }
      phif[v] = 0.5 * (phiL + phiR);
      // Eq. (AD-eqn3): chain rule with the interpolated unhatted metrics
      for (int a = 0; a < nd; ++a) {
        real s = 0.0;
        for (int e = 0; e < nd; ++e) s = s + g.fu[d][e][a].at(i, j, k) * gc[e];
        gx[v][a] = s;
      }
    }
    real mu = viscosity(phif[nd]);
    real lam = -2.0 / 3.0 * mu;
    real kap = mu * gamma / ((gamma - 1.0) * p.prandtl);
    real div = 0.0;
    for (int a = 0; a < nd; ++a) div = div + gx[a][a];
    real tau[3][3], beta[3];
    for (int a = 0; a < nd; ++a)
      for (int b = 0; b < nd; ++b) {
        tau[a][b] = mu * (gx[a][b] + gx[b][a]);  // Eq. (shear-str)
        if (a == b) tau[a][b] = tau[a][b] + lam * div;
      }
    for (int a = 0; a < nd; ++a) {
      real s = 0.0;
      for (int b = 0; b < nd; ++b) s = s + phif[b] * tau[a][b];
      beta[a] = s + kap * gx[nd][a];  // Eq. (thermal-work)
    }
    real Fv[5];
    Fv[0] = 0.0;
    for (int a = 0; a < nd; ++a) {
      real s = 0.0;
      for (int b = 0; b < nd; ++b) s = s + nh[b] * tau[a][b];
      Fv[1 + a] = s;
    }
    {
      real s = 0.0;
      for (int b = 0; b < nd; ++b) s = s + nh[b] * beta[b];
      Fv[nv - 1] = s;
    }
    for (int c = 0; c < nv; ++c) F[c] = F[c] - Fv[c];
  }
  for (int c = 0; c < nv; ++c) G[c] = F[c];
#undef CELL
}

int orc_solver::rhs(const double* q, double* Lout, double* resout, int fdir, double* gout, double* primout) {
  const size_t NC = inner.size();
  Field P[5];
  for (int c = 0; c < nv; ++c) P[c] = Field(pad);
  // primitive variables at the cell centres (Sec. 2)
  ORC_PHASE(PH_PRIM);
  const real gm1 = p.gamma - 1.0;
  FOR_BOX(inner) {
    size_t id = inner.idx(i, j, k);
    real rho = q[id];
    real ke = 0.0;
    P[0].at(i, j, k) = rho;
    for (int a = 0; a < nd; ++a) {
      real ua = q[(size_t)(1 + a) * NC + id] / rho;
      P[1 + a].at(i, j, k) = ua;
      ke = ke + ua * ua;
    }
    real En = q[(size_t)(nv - 1) * NC + id];
    P[nv - 1].at(i, j, k) = gm1 * (En - 0.5 * rho * ke);
  }
  fill_ghosts(P);
  if (primout) {
    for (int c = 0; c < nv; ++c) {
      FOR_BOX(inner) { primout[(size_t)c * NC + inner.idx(i, j, k)] = Dbl(P[c].at(i, j, k)); }
    }
  }
  Field T;
  if (viscous) {
    T = Field(pad);
    FOR_BOX(pad) { T.at(i, j, k) = P[nv - 1].at(i, j, k) / P[0].at(i, j, k); }  // T = p/rho (gas constant R = 1)
  }
  // Sec. 5.1 step 1: gradients along each computational direction
  ORC_PHASE(PH_GRAD);
  Field P1[3][5], P2[3][5], T1[3];
  const bool mig4 = p.gradient_scheme == 1;
  for (int d = 0; d < nd; ++d) {
    for (int c = 0; c < nv; ++c) {
      P1[d][c] = mig4 ? op_ig4(P[c], d, p.periodic[d] != 0, p.n[d]) : op_e6(P[c], d);
      P2[d][c] = op_second(P[c], P1[d][c], d);
    }
    if (viscous) T1[d] = mig4 ? op_ig4(T, d, p.periodic[d] != 0, p.n[d]) : op_e6(T, d);
  }
  // interface fluxes G = F^ - F^v for faces i+1/2, i = -1..n-1
  ORC_PHASE(PH_FACE);
  Field Gf[3][5];
  for (int d = 0; d < nd; ++d) {
    Box fb = inner;
    fb.lo[d] = -1;
    fb.hi[d] = p.n[d];
    for (int c = 0; c < nv; ++c) Gf[d][c] = Field(fb);
    FOR_BOX(fb) {
      real G[5];
      face_flux(d, i, j, k, P, P1, P2, T, T1, G);
      for (int c = 0; c < nv; ++c) Gf[d][c].at(i, j, k) = G[c];
    }
  }
  if (gout) {
    Box fb = inner;
    fb.lo[fdir] = -1;
    fb.hi[fdir] = p.n[fdir];
    for (int c = 0; c < nv; ++c) {
      size_t m = 0;
      for (int k = fb.lo[2]; k < fb.hi[2]; ++k)
        for (int j = fb.lo[1]; j < fb.hi[1]; ++j)
          for (int i = fb.lo[0]; i < fb.hi[0]; ++i) gout[(size_t)c * fb.size() + (m++)] = Dbl(Gf[fdir][c].at(i, j, k));
    }
  }
  // Sec. 3: Res = -sum_d [(F^ - F^v)_{+1/2} - (F^ - F^v)_{-1/2}]; time split of Sec. 4
  ORC_PHASE(PH_RES);
  for (int c = 0; c < nv; ++c) {
    FOR_BOX(inner) {
      size_t id = inner.idx(i, j, k);
      real res = 0.0;
      for (int d = 0; d < nd; ++d) res = res - (Gf[d][c].at(i, j, k) - Gf[d][c].sh(i, j, k, d, -1));
      if (resout) resout[(size_t)c * NC + id] = Dbl(res);
      if (Lout) {
        real J = 1.0 / g.det.at(i, j, k);
        real qc = q[(size_t)c * NC + id];
        real L = g.moving ? J * (res - g.gcl.at(i, j, k) * qc) : J * res;
        if (!sigma.empty()) L = L - sigma[id] * (qc - qamb[c]);  // sponge source
        Lout[(size_t)c * NC + id] = Dbl(L);
      }
    }
  }
  ORC_PHASE(PH_MISC);
  return 0;
}

// ---------------------------------------------------------------------------
// C API
// ---------------------------------------------------------------------------
extern "C" {

const char* orc_last_error(void) { return g_err.c_str(); }
int orc_ext_pad(void) { return E; }
int orc_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int orc_create(const orc_params* prm, const double* nodes, const double* node_vel, orc_solver** out) {
  *out = nullptr;
  if (!prm || (prm->ndim != 2 && prm->ndim != 3)) return fail("ndim must be 2 or 3");
  orc_solver* s = new orc_solver();
  s->p = *prm;
  s->nd = prm->ndim;
  s->nv = prm->ndim + 2;
  if (s->nd == 2) s->p.n[2] = 1;
  for (int d = 0; d < s->nd; ++d) {
    if (s->p.n[d] < H && s->p.periodic[d]) { delete s; return fail("periodic axis needs at least 6 cells"); }
    if (s->p.n[d] < 1) { delete s; return fail("empty axis"); }
    if (!s->p.periodic[d] && s->p.ghost_nodes != 0 && s->p.ghost_nodes < E) {
      delete s;
      return fail("non-periodic axis needs >= 10 ghost node layers, or none (App. C)");
    }
    if (!s->p.periodic[d] && s->p.ghost_nodes == 0 && s->p.n[d] < 2 * H) {
      delete s;
      return fail("an axis without ghost nodes needs at least 12 cells");
    }
    if (!s->p.periodic[d] && s->p.ghost_nodes == 0 && node_vel) {
      delete s;
      return fail("moving meshes need ghost nodes on non-periodic axes");
    }
    for (int side = 0; side < 2; ++side)
      if (!s->p.periodic[d] && s->p.bc[d][side] == ORC_BC_WALL && s->p.n[d] < H) {
        delete s;
        return fail("a wall axis needs at least 6 cells");
      }
  }
  s->viscous = prm->reynolds > 0.0;
  s->inner = make_box(s->nd, s->p.n, 0);
  s->pad = make_box(s->nd, s->p.n, H);
  s->ext = make_box(s->nd, s->p.n, E);
  s->cellgeo = make_box(s->nd, s->p.n, 5);
  for (int d = 0; d < s->nd; ++d) {
    s->closed[d] = !s->p.periodic[d] && s->p.ghost_nodes == 0;
    if (s->closed[d]) {  // geometry exists on the cells only
      s->ext.lo[d] = s->cellgeo.lo[d] = 0;
      s->ext.hi[d] = s->cellgeo.hi[d] = s->p.n[d];
    } else if (s->p.periodic[d] && s->p.gradient_scheme == 1 && s->p.metric_scheme == 0) {
      // MIG4 metrics: long unwrapped lines on periodic axes (see op_interp_ig4)
      s->ext.lo[d] = -kExtIG4;
      s->ext.hi[d] = s->p.n[d] + kExtIG4;
      s->cellgeo.lo[d] = -kCellIG4;
      s->cellgeo.hi[d] = s->p.n[d] + kCellIG4;
    }
  }
  s->inflow.assign((size_t)s->nv * s->p.n[1] * s->p.n[2], 0.0);
  if (nodes) {
    int rc = orc_set_nodes(s, nodes, node_vel);
    if (rc) { delete s; return rc; }
  }
  *out = s;
  return 0;
}

int orc_set_nodes(orc_solver* s, const double* nodes, const double* node_vel) {
  Field xc[3], vc[3];
  int rc = s->centroids_from_nodes(nodes, node_vel, xc, vc);
  if (rc) return rc;
  return s->build_geometry(xc, node_vel ? vc : nullptr);
}

int orc_set_centroids(orc_solver* s, const double* xc_ext, const double* vc_ext) {
  Field xc[3], vc[3];
  const size_t NE = s->ext.size();
  for (int a = 0; a < s->nd; ++a) {
    xc[a] = Field(s->ext);
    for (size_t m = 0; m < NE; ++m) xc[a].v[m] = xc_ext[a * NE + m];
    if (vc_ext) {
      vc[a] = Field(s->ext);
      for (size_t m = 0; m < NE; ++m) vc[a].v[m] = vc_ext[a * NE + m];
    }
  }
  return s->build_geometry(xc, vc_ext ? vc : nullptr);
}

void orc_destroy(orc_solver* s) { delete s; }

static void copy_out(const Field& f, const Box& b, double* out) {
  size_t m = 0;
  for (int k = b.lo[2]; k < b.hi[2]; ++k)
    for (int j = b.lo[1]; j < b.hi[1]; ++j)
      for (int i = b.lo[0]; i < b.hi[0]; ++i) out[m++] = Dbl(f.at(i, j, k));
}

void orc_get_cell_metrics(const orc_solver* s, double* mh, double* det) {
  const size_t NC = s->inner.size();
  for (int e = 0; e < s->nd; ++e)
    for (int a = 0; a < s->nd; ++a)
      if (mh) copy_out(s->g.mh[e][a], s->inner, mh + (size_t)(e * s->nd + a) * NC);
  if (det) copy_out(s->g.det, s->inner, det);
}

void orc_get_cell_time_metrics(const orc_solver* s, double* mt) {
  const size_t NC = s->inner.size();
  for (int e = 0; e < s->nd; ++e) {
    if (s->g.moving) copy_out(s->g.mt[e], s->inner, mt + (size_t)e * NC);
    else for (size_t m = 0; m < NC; ++m) mt[(size_t)e * NC + m] = 0.0;
  }
}

void orc_get_face_metrics(const orc_solver* s, int d, double* fh, double* fu, double* ft) {
  Box fb = s->inner;
  fb.lo[d] = -1;
  fb.hi[d] = s->p.n[d];
  const size_t NF = fb.size();
  for (int a = 0; a < s->nd; ++a)
    if (fh) copy_out(s->g.fh[d][a], fb, fh + (size_t)a * NF);
  if (fu && s->viscous)
    for (int e = 0; e < s->nd; ++e)
      for (int a = 0; a < s->nd; ++a) copy_out(s->g.fu[d][e][a], fb, fu + (size_t)(e * s->nd + a) * NF);
  if (ft) {
    if (s->g.moving) copy_out(s->g.ft[d], fb, ft);
    else for (size_t m = 0; m < NF; ++m) ft[m] = 0.0;
  }
}

void orc_get_gcl(const orc_solver* s, double* gcl) { copy_out(s->g.gcl, s->inner, gcl); }

void orc_set_inflow(orc_solver* s, const double* prim) {
  for (size_t m = 0; m < s->inflow.size(); ++m) s->inflow[m] = prim[m];
}

void orc_set_sponge(orc_solver* s, const double* sigma, const double* q_amb) {
  if (!sigma) { s->sigma.clear(); s->qamb.clear(); return; }
  s->sigma.assign(sigma, sigma + s->inner.size());
  s->qamb.assign(q_amb, q_amb + s->nv);
}

int orc_rhs(orc_solver* s, const double* q, double* L) { return s->rhs(q, L, nullptr, 0, nullptr, nullptr); }
int orc_residual(orc_solver* s, const double* q, double* res) { return s->rhs(q, nullptr, res, 0, nullptr, nullptr); }
int orc_face_flux(orc_solver* s, const double* q, int d, double* gout) {
  if (d < 0 || d >= s->nd) return fail("bad direction");
  return s->rhs(q, nullptr, nullptr, d, gout, nullptr);
}
int orc_primitives(orc_solver* s, const double* q, double* prim) {
  return s->rhs(q, nullptr, nullptr, 0, nullptr, prim);
}

// App. B: dt = CFL * min over cells and directions of 1/(|U| + c |grad xi|),
// with the viscous bound 1 / (nu_eff |grad xi|^2), nu_eff = max(4/3, gamma/Pr) mu / rho, when the flow is viscous.
double orc_dt(orc_solver* s, const double* q, double cfl) {
  const int nd = s->nd, nv = s->nv;
  const size_t NC = s->inner.size();
  real best = std::numeric_limits<double>::infinity();
  const real gamma = s->p.gamma;
  const Box& B = s->inner;
  for (int k = B.lo[2]; k < B.hi[2]; ++k)
    for (int j = B.lo[1]; j < B.hi[1]; ++j)
      for (int i = B.lo[0]; i < B.hi[0]; ++i) {
        size_t id = B.idx(i, j, k);
        real rho = q[id];
        real u[3], ke = 0.0;
        for (int a = 0; a < nd; ++a) {
          u[a] = q[(size_t)(1 + a) * NC + id] / rho;
          ke = ke + u[a] * u[a];
        }
        real pr = (gamma - 1.0) * (q[(size_t)(nv - 1) * NC + id] - 0.5 * rho * ke);
        real c = Sqrt(gamma * pr / rho);
        real J = 1.0 / s->g.det.at(i, j, k);
        for (int e = 0; e < nd; ++e) {
          real U = s->g.moving ? s->g.mt[e].at(i, j, k) * J : real(0.0);
          real g2 = 0.0;
          for (int a = 0; a < nd; ++a) {
            real m = s->g.mh[e][a].at(i, j, k) * J;  // unhatted metric
            U = U + m * u[a];
            g2 = g2 + m * m;
          }
          real gn = Sqrt(g2);
          best = Min(best, 1.0 / (Fabs(U) + c * gn));
          if (s->viscous) {
            real mu = s->viscosity(pr / rho);
            real fac = (4.0 / 3.0 > gamma / s->p.prandtl) ? real(4.0 / 3.0) : gamma / s->p.prandtl;
            real nu = fac * mu / rho;
            best = Min(best, 1.0 / (nu * g2));
          }
        }
      }
  return Dbl(cfl * best);
}

double orc_viscosity(const orc_solver* s, double T) { return Dbl(s->viscosity(real(T))); }

// App. B: three-stage SSP (TVD) Runge-Kutta, advancing Q with L(Q) = J (Res - (1/J)_t Q).
int orc_rk3(orc_solver* s, double* q, double dt, const double* const* stage_nodes, const double* const* stage_vel) {
  const size_t N = (size_t)s->nv * s->inner.size();
  std::vector<double> q0(q, q + N), q1(N), q2(N), L(N);
  int rc;
  if (stage_nodes && (rc = orc_set_nodes(s, stage_nodes[0], stage_vel ? stage_vel[0] : nullptr))) return rc;
  s->rhs(q0.data(), L.data(), nullptr, 0, nullptr, nullptr);
  for (size_t m = 0; m < N; ++m) q1[m] = Dbl(real(q0[m]) + real(dt) * real(L[m]));
  if (stage_nodes && (rc = orc_set_nodes(s, stage_nodes[1], stage_vel ? stage_vel[1] : nullptr))) return rc;
  s->rhs(q1.data(), L.data(), nullptr, 0, nullptr, nullptr);
  for (size_t m = 0; m < N; ++m)
    q2[m] = Dbl(0.75 * real(q0[m]) + 0.25 * real(q1[m]) + 0.25 * real(dt) * real(L[m]));
  if (stage_nodes && (rc = orc_set_nodes(s, stage_nodes[2], stage_vel ? stage_vel[2] : nullptr))) return rc;
  s->rhs(q2.data(), L.data(), nullptr, 0, nullptr, nullptr);
  for (size_t m = 0; m < N; ++m)
    q[m] = Dbl((1.0 / 3.0) * real(q0[m]) + (2.0 / 3.0) * real(q2[m]) + (2.0 / 3.0) * real(dt) * real(L[m]));
  return 0;
}

void orc_op1d(int kind, int n, const double* f, double* out) {
  Box b;
  b.lo[0] = -E; b.hi[0] = n + E;
  b.lo[1] = b.lo[2] = 0; b.hi[1] = b.hi[2] = 1;
  Field F(b);
  for (int i = -E; i < n + E; ++i) F.at(i, 0, 0) = f[((i % n) + n) % n];
  Field o;
  switch (kind) {
    case 0: o = op_e6(F, 0); break;
    case 1: o = op_second(F, op_e6(F, 0), 0); break;
    case 2: o = op_interp(F, 0, 0); break;
    case 3: o = op_D(F, 0); break;
    case 4: o = op_e4(F, 0); break;
    case 5: o = op_ig4(F, 0, true, n); break;
    case 7: {
      // the App. C derivative D on a wall-bounded line: the values themselves, no wrap
      Box cb;
      cb.lo[0] = 0; cb.hi[0] = n;
      cb.lo[1] = cb.lo[2] = 0; cb.hi[1] = cb.hi[2] = 1;
      Field C(cb);
      for (int i = 0; i < n; ++i) C.at(i, 0, 0) = f[i];
      Field D = op_delta(op_interp_c(C, 0), 0);
      for (int i = 0; i < n; ++i) out[i] = Dbl(D.at(i, 0, 0));
      return;
    }
    default: {
      // open line: the values themselves, no wrap
      std::vector<real> line(f, f + n), g;
      ig4_line_open(line.data(), n, g);
      for (int i = 0; i < n; ++i) out[i] = Dbl(g[i]);
      return;
    }
  }
  for (int i = 0; i < n; ++i) out[i] = Dbl(o.at(i, 0, 0));
}

void orc_eigen(int nd, const double* nh, double rho, double p, double gamma, double* R, double* Rinv) {
  real n[3] = {nh[0], nh[1], nd == 3 ? nh[2] : 0.0};
  real Rm[5][5], Lm[5][5];
  eigen(nd, n, rho, p, gamma, Rm, Lm);
  const int nv = nd + 2;
  for (int r = 0; r < nv; ++r)
    for (int c = 0; c < nv; ++c) {
      R[r * nv + c] = Dbl(Rm[r][c]);
      Rinv[r * nv + c] = Dbl(Lm[r][c]);
    }
}

void orc_hllc(int nd, const double* PL, const double* PR, const double* nh, double nt, double gamma, double* F) {
  const int nv = nd + 2;
  real pl[5] = {0.0, 0.0, 0.0, 0.0, 0.0}, pr[5] = {0.0, 0.0, 0.0, 0.0, 0.0}, n[3] = {0.0, 0.0, 0.0}, f[5];
  for (int c = 0; c < nv; ++c) { pl[c] = PL[c]; pr[c] = PR[c]; }
  for (int a = 0; a < nd; ++a) n[a] = nh[a];
  hllc(nd, pl, pr, n, nt, gamma, f);
  for (int c = 0; c < nv; ++c) F[c] = Dbl(f[c]);
}

double orc_mp_limit(double wface, double w_up, double w_base, double w_down, double d_up, double d_base,
                    double d_down, double alpha, double beta, double eps) {
  return Dbl(mp_limit(wface, w_up, w_base, w_down, d_up, d_base, d_down, alpha, beta, eps));
}

void orc_count_reset(void) {
#ifdef ORC_COUNTING
  for (int m = 0; m < 8; ++m) orc_counters[m] = OrcCounters{0, 0, 0, 0};
  orc_phase = PH_MISC;
#endif
}
void orc_count_get(unsigned long long* add, unsigned long long* mul, unsigned long long* div, unsigned long long* sq) {
  orc_count_get_phase(-1, add, mul, div, sq);
}
void orc_count_get_phase(int phase, unsigned long long* add, unsigned long long* mul, unsigned long long* div,
                         unsigned long long* sq) {
  *add = *mul = *div = *sq = 0;
#ifdef ORC_COUNTING
  for (int m = 0; m < 8; ++m) {
    if (phase >= 0 && m != phase) continue;
    *add += orc_counters[m].add; *mul += orc_counters[m].mul; *div += orc_counters[m].div; *sq += orc_counters[m].sqrt;
  }
#else
  (void)phase;
#endif
}
int orc_is_counting(void) {
#ifdef ORC_COUNTING
  return 1;
#else
  return 0;
#endif
}

}  // extern "C"
