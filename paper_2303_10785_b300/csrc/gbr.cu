// sm_103a library: kernels and the C ABI declared in include/gbr.h.
//
// Per RK stage (FP64, or the mixed path's FP32 where gbr_params.precision says;
// every step of the path in these kernels):
//   k_prim_halo (primitives and all ghost layers in one pass) -> k_grad1 (E6;
//   MIG4: k_ig4, one launch per direction) -> k_grad2 -> k_face (one launch per
//   direction) -> k_update (divergence, GCL term, sponge, SSP-RK3 combination)
// Geometry (set-up, or every stage of a moving mesh):
//   k_motion -> k_centroid -> k_coordd -> k_metrics -> k_face_metrics -> k_gcl
// Time step: k_dt (block min with warp shuffles + atomicMin on the bits of a
// positive double) -> k_dt_final.  dt and t stay on the device.
#include <cuda.h>
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "../../include/gbr.h"
#include "gbr_kernels.cuh"

using namespace gbr;

namespace {

// Launch shape of the interface kernel (tuning knobs, set at compile time).  The FP64
// instantiations are FP64-pipe bound and run 4 blocks of 128 threads per SM (at most 128
// registers: unbounded, the viscous one takes 130-132 and only 3 blocks fit); the FP32 ones are
// issue- and latency-bound and run 7 blocks per SM (72 registers; measured on the 128^3 TGV:
// 6 blocks / 80 registers 5 % slower, 8 / 64 spills, unconstrained 128 registers 17 % slower).
#ifndef GBR_FACE_BLOCK
#define GBR_FACE_BLOCK 128
#endif
#ifndef GBR_FACE_MIN_BLOCKS
#define GBR_FACE_MIN_BLOCKS 4
#endif
#ifndef GBR_FACE_MIN_BLOCKS_F32
#define GBR_FACE_MIN_BLOCKS_F32 7
#endif
// The 3D x-sweep: its own block shape (the same by default; 256 threads x 2 blocks per SM measured
// slower in both precisions), and its warps' interfaces.  Along x an extremum of the flow is a point,
// so 32 consecutive x-interfaces hold a few interfaces that fail the App. E test, and every warp
// pays for queueing them; with GBR_FACE_XT_WX = WX > 0 a warp holds WX consecutive x-interfaces of
// 32 / WX consecutive y-lines instead, so that failing interfaces fill whole warps as they do in the
// y- and z-sweeps, at the price of strided loads (each lane its own y-line).  FP64 (pipe-bound,
// loads far from the bound): WX = 1, 128^3 TGV step 16.64 -> 16.38 ms (WX = 2: 16.41, 4: 16.62).
// FP32 (issue- and latency-bound): the linear mapping (WX = 8 / 16 / 32: 1.83 / 1.88 / 1.99 ms
// per step against 1.80).
#ifndef GBR_FACE_BLOCK_X
#define GBR_FACE_BLOCK_X GBR_FACE_BLOCK
#endif
#ifndef GBR_FACE_MIN_BLOCKS_X
#define GBR_FACE_MIN_BLOCKS_X GBR_FACE_MIN_BLOCKS
#endif
#ifndef GBR_FACE_MIN_BLOCKS_F32_X
#define GBR_FACE_MIN_BLOCKS_F32_X GBR_FACE_MIN_BLOCKS_F32
#endif
#ifndef GBR_FACE_XT_WX
#define GBR_FACE_XT_WX 1
#endif
#ifndef GBR_FACE_XT_WX_F32
#define GBR_FACE_XT_WX_F32 0
#endif

constexpr int kBlock = 256;

enum { S_DT = 0, S_T = 1, S_DTMIN = 2, S_NSCAL = 8 };

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
#define BOX_THREAD(B)                                                   \
  const long long _t = (long long)blockIdx.x * blockDim.x + threadIdx.x; \
  if (_t >= box_size(B)) return;                                       \
  int i, j, k;                                                          \
  box_coord(B, _t, i, j, k);

__global__ void k_motion(Layout L, Motion M, const double* scal, double stage_c, double* nodes, double* nvel,
                         Box b) {
  BOX_THREAD(b);
  const double tau = scal[S_T] + stage_c * scal[S_DT];
  const double ph = 2.0 * M.omega * tau;  // sin(2 pi omega tau) = sinpi(2 omega tau)
  const double st = sinpi(ph);
  const double ct = 2.0 * 3.14159265358979323846 * M.omega * cospi(ph);
  body_motion(L, M, st, ct, nodes, nvel, i, j, k);
}

__global__ void k_centroid(GeoArgs G, Box b) {
  BOX_THREAD(b);
  body_centroid(G, i, j, k);
}

__global__ void k_coordd(GeoArgs G, Box b0, Box b1, Box b2) {
  const int d = blockIdx.y;
  const Box b = d == 0 ? b0 : (d == 1 ? b1 : b2);
  BOX_THREAD(b);
  body_coord_derivative(G, d, i, j, k);
}

__global__ void k_metrics(GeoArgs G, Box b) {
  BOX_THREAD(b);
  body_metrics(G, i, j, k);
}

__global__ void k_face_metrics(GeoArgs G, Box b0, Box b1, Box b2) {
  const int d = blockIdx.y;
  const Box b = d == 0 ? b0 : (d == 1 ? b1 : b2);
  BOX_THREAD(b);
  body_face_metrics(G, d, i, j, k);
}

// the FP64 path's interface geometry from the interface metrics (body_face_geo)
struct FaceGeoOut {
  double* fg[3];
};
__global__ void k_face_geo(GeoArgs G, FaceGeoOut O, Box b0, Box b1, Box b2) {
  const int d = blockIdx.y;
  const Box b = d == 0 ? b0 : (d == 1 ? b1 : b2);
  BOX_THREAD(b);
  body_face_geo(G, O.fg[d], d, i, j, k);
}

// ---- MIG4 metrics: one thread per geometry line (set-up work; Sec. 7 step 2 with IG4)
__global__ void k_ig4_geo_factor(double* t, int m) { ig4_geo_factor(t, m); }

// D_d of one direction on its own (the App. C closure of a wall-bounded axis of a MIG4 grid)
__global__ void k_coordd1(GeoArgs G, int d, Box b) {
  BOX_THREAD(b);
  body_coord_derivative(G, d, i, j, k);
}

// xd[a][d] = D_d(x_a) on [-he + 5, n + he - 5) along d; xs: cross-section of the extended box
__global__ void k_ig4_coordd(GeoArgs G, int d, Box xs, const double* t, double* w) {
  BOX_THREAD(xs);
  const Layout& L = G.L;
  const long long base = line_base(L, d, i, j, k), st = L.es[d];
  const int lo = -L.he[d], hi = L.n[d] + L.he[d];
  const LineRef W{w + base, st};
  for (int a = 0; a < L.nd; ++a) {
    const double* x = G.xc + a * L.ecount + base;
    auto f = [&](int m) { return x[m * st]; };
    ig4_geo_solve(f, W, lo, hi, t);
    double* out = G.xd + (a * 3 + d) * L.ecount + base;
    double prev = ig4_geo_face(f, W, lo + 4);
    for (int m = lo + 5; m < hi - 5; ++m) {
      const double cur = ig4_geo_face(f, W, m);
      out[m * st] = cur - prev;
      prev = cur;
    }
  }
}

// Eq. (GCL_metrics), 3D, the derivatives along s: phase 0 stores, for e = s + 1, the term
// D_s(x_b,f x_c) with f = s + 2; phase 1 subtracts, for e = s + 2, the term D_s(x_b,g x_c) with
// g = s + 1 (b = a + 1, c = a + 2).  xs: cross-section of the cell-metric box.
__global__ void k_ig4_metric_terms(GeoArgs G, int s, int phase, Box xs, const double* t, double* w) {
  BOX_THREAD(xs);
  const Layout& L = G.L;
  const long long EC = L.ecount;
  const long long base = line_base(L, s, i, j, k), st = L.es[s];
  const int lo = -L.he[s], hi = L.n[s] + L.he[s];
  const int olo = -L.cg[s], ohi = L.n[s] + L.cg[s];
  const int e = phase == 0 ? (s + 1) % 3 : (s + 2) % 3;
  const int inner = phase == 0 ? (s + 2) % 3 : (s + 1) % 3;  // the coordinate derivative in the product
  const LineRef W{w + base, st};
  for (int a = 0; a < 3; ++a) {
    const int b = (a + 1) % 3, c = (a + 2) % 3;
    const double* u = G.xd + (b * 3 + inner) * EC + base;
    const double* v = G.xc + c * EC + base;
    auto f = [&](int m) { return u[m * st] * v[m * st]; };
    double* out = G.mh + (e * 3 + a) * EC + base;
    if (L.closed[s]) {
      for (int m = 0; m < L.n[s]; ++m) {
        const double dv = appc_D(f, m, L.n[s]);
        out[m * st] = phase == 0 ? dv : out[m * st] - dv;
      }
      continue;
    }
    ig4_geo_solve(f, W, lo, hi, t);
    double prev = ig4_geo_face(f, W, olo - 1);
    for (int m = olo; m < ohi; ++m) {
      const double cur = ig4_geo_face(f, W, m);
      const double dv = cur - prev;
      out[m * st] = phase == 0 ? dv : out[m * st] - dv;
      prev = cur;
    }
  }
}

// 1/J, unhatted and time metrics from the coordinate derivatives and the hat metrics
__global__ void k_metrics_given(GeoArgs G, Box b) {
  BOX_THREAD(b);
  body_metrics(G, i, j, k, true);
}

// Sec. 7 step 3 with IG4: interface metrics of direction d, one line of the cell-metric box per
// thread (xs: the cross-section of the interior)
__global__ void k_ig4_face_metrics(GeoArgs G, int d, Box xs, const double* t, double* w) {
  BOX_THREAD(xs);
  const Layout& L = G.L;
  const long long EC = L.ecount, FC = L.fcount[d];
  const long long base = line_base(L, d, i, j, k), st = L.es[d];
  const int lo = -L.cg[d], hi = L.n[d] + L.cg[d];
  const int nd = L.nd;
  const LineRef W{w + base, st};
  int c0[3] = {i, j, k};
  c0[d] = 0;
  const long long f0 = fidx(L, d, c0[0], c0[1], c0[2]), fs = L.fs[d][d];  // interface 1/2; -1/2 at f0 - fs
  auto interp = [&](const double* src, double* dst) {
    const double* x = src + base;
    auto f = [&](int m) { return x[m * st]; };
    if (L.closed[d]) {
      for (int m = -1; m < L.n[d]; ++m) dst[f0 + m * fs] = appc_face(f, m, L.n[d]);
      return;
    }
    ig4_geo_solve(f, W, lo, hi, t);
    for (int m = -1; m < L.n[d]; ++m) dst[f0 + m * fs] = ig4_geo_face(f, W, m);
  };
  for (int a = 0; a < nd; ++a) interp(G.mh + (d * 3 + a) * EC, G.fh[d] + a * FC);
  if (G.viscous)
    for (int ee = 0; ee < nd; ++ee)
      for (int a = 0; a < nd; ++a) interp(G.mu + (ee * 3 + a) * EC, G.fu[d] + (ee * nd + a) * FC);
  if (G.moving) interp(G.mt + d * EC, G.ft[d]);
}

__global__ void k_gcl(GeoArgs G, Box b) {
  BOX_THREAD(b);
  body_gcl(G, i, j, k);
}

template <int ND, class R = double>
__global__ void k_prim(RhsArgsT<R> A, Box b) {
  BOX_THREAD(b);
  body_prim<ND>(A, i, j, k);
}

// Primitive and update passes: latency-bound streams, run at full occupancy (8 blocks of 256 threads
// per SM, 32 registers): the mixed 128^3 TGV step 4.7 % faster than at 42 / 54 registers.
constexpr int kStreamBlocks = 8;

template <int ND, class R = double, bool SPECIAL = true>
__global__ void __launch_bounds__(kBlock, kStreamBlocks) k_prim_halo(RhsArgsT<R> A, const double* q,
                                                                     const float* dq, Box b) {
  BOX_THREAD(b);
  body_prim_halo<ND, R, SPECIAL>(A, q, dq, i, j, k);
}

template <int ND, class R = double>
__global__ void k_halo(RhsArgsT<R> A, int d, Box b) {
  BOX_THREAD(b);
  body_halo<ND>(A, d, i, j, k);
}

// Gradient passes: the ND directions of one chunk of cells are consecutive blocks, so the passes
// over a chunk run close together in time and share its fields in L2 (one DRAM read of each
// field instead of one per direction).
#define GRAD_THREAD(B0, B1, B2)                                                   \
  const int e = blockIdx.x % ND;                                                  \
  const Box b = e == 0 ? B0 : (e == 1 ? B1 : B2);                                 \
  const long long _t = (long long)(blockIdx.x / ND) * blockDim.x + threadIdx.x;   \
  if (_t >= box_size(b)) return;                                                  \
  int i, j, k;                                                                    \
  box_coord(b, _t, i, j, k);

template <int ND, class R = double>
__global__ void k_grad1(RhsArgsT<R> A, Box b0, Box b1, Box b2) {
  GRAD_THREAD(b0, b1, b2);
  body_grad1<ND>(A, e, i, j, k);
}

// E6 first derivatives of one field in all three directions, 3D (Eq. 11), by a block that owns a
// 32 x 8 tile of (x, y) columns and marches along z through a chunk of planes.  Each column keeps
// its seven values z-3 .. z+3 in registers (the z-derivative, one new load per plane); each plane
// goes to shared memory with a ring of 3 cells around the tile (the x- and y-derivatives), written
// from the columns' centre values plus the ring loads, double-buffered so that one barrier per
// plane suffices.  Every value is read from global memory about once per plane (the ring and the
// chunk ends aside) instead of once per stencil point, and the three derivatives are stored with
// consecutive threads on consecutive x.  Outputs and arithmetic are those of body_grad1 on the
// three first-derivative boxes (each cell of a box gets exactly its stencil_E6x60 value).  The
// per-cell kernel was issue-bound on index arithmetic (53 instructions per derivative, 62 % of
// the issue slots busy); running pointers and one ring load per thread and plane take the 128^3
// mixed step from 1.929 to 1.874 ms.
constexpr int kG1TX = 32, kG1TY = 8, kG1Ring = 3;
constexpr int kG1SX = kG1TX + 2 * kG1Ring, kG1SY = kG1TY + 2 * kG1Ring;
constexpr int kG1RingCount = kG1SX * kG1SY - kG1TX * kG1TY;  // 276

// (row, column) in the plane tile of the r-th ring cell: the top rows, the sides of the middle
// rows, the bottom rows
__device__ __forceinline__ void g1_ring_pos(int r, int& sy, int& sx) {
  constexpr int top = kG1Ring * kG1SX, side = 2 * kG1Ring;
  if (r < top) {
    sy = r / kG1SX;
    sx = r % kG1SX;
  } else if (r < top + kG1TY * side) {
    const int q = r - top;
    sy = kG1Ring + q / side;
    const int c = q % side;
    sx = c < kG1Ring ? c : kG1TX + c;
  } else {
    const int q = r - top - kG1TY * side;
    sy = kG1Ring + kG1TY + q / kG1SX;
    sx = q % kG1SX;
  }
}

constexpr int kG1Waves = 3;
constexpr int kG1Fields = 1;  // fields per block (2 and 3, one barrier per plane for all, measured no faster)

// streaming multiprocessors of the current device (queried once)
inline int device_sms() {
  static int v = 0;
  if (v < 1) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        v < 1)
      v = 148;
  }
  return v;
}

template <class R, int FPB>
__global__ void __launch_bounds__(kG1TX * kG1TY) k_grad1t(RhsArgsT<R> A, Box U, Box bx, Box by, Box bz, int tiles_x,
                                                          int tiles_y, int zchunk, int nf) {
  constexpr int NV = 5;
  constexpr int PL = kG1SX * kG1SY;  // one plane tile
  __shared__ R plane[2][FPB][PL];
  const Layout& L = A.L;
  const int tid = threadIdx.x, tx = tid % kG1TX, ty = tid / kG1TX;
  const int t = blockIdx.x;
  const int tlx = t % tiles_x, tly = (t / tiles_x) % tiles_y, chunk = t / (tiles_x * tiles_y);
  const int x0 = U.lo[0] + tlx * kG1TX, y0 = U.lo[1] + tly * kG1TY;  // cell of tile point (0, 0)
  const int x = x0 + tx, y = y0 + ty;
  const int zs = U.lo[2] + chunk * zchunk, ze = min(zs + zchunk, U.hi[2]);
  const long long PC = L.pcount, sz = L.ps[2];
  // fields f0 .. f0 + FPB - 1 of this block (the last block of an odd count repeats the last
  // field: same values written twice)
  const R* src[FPB];
  long long fo[FPB];
#pragma unroll
  for (int q = 0; q < FPB; ++q) {
    const int f = min(blockIdx.y * FPB + q, nf - 1);
    src[q] = (f < NV) ? A.prim + f * PC : A.temp;
    fo[q] = f * PC;
  }
  // A value is loaded only where its (x, y) lies in the padded box (outside it no output needs
  // it).  Along z no check is needed: the planes read, zs - 3 .. ze + 2 with zs >= -3 and
  // ze <= n_z + 3, lie in the padded range -H .. n_z + H - 1.
  auto inside = [&](int cx, int cy) {
    return cx >= -L.hp[0] && cx < L.n[0] + L.hp[0] && cy >= -L.hp[1] && cy < L.n[1] + L.hp[1];
  };
  const bool col = inside(x, y);
  const long long pcol = col ? pidx(L, x, y, 0) : 0;  // padded index of (x, y, 0)
  // the ring cells this thread loads (at most two): shared-memory slot and padded offset
  int r_off[2];
  bool r_ok[2];
  long long r_p[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int r = tid + h * kG1TX * kG1TY;
    int sy = 0, sx = 0;
    r_ok[h] = false;
    if (r < kG1RingCount) {
      g1_ring_pos(r, sy, sx);
      r_ok[h] = inside(x0 + sx - kG1Ring, y0 + sy - kG1Ring);
    }
    r_off[h] = (r < kG1RingCount) ? sy * kG1SX + sx : -1;
    r_p[h] = r_ok[h] ? pidx(L, x0 + sx - kG1Ring, y0 + sy - kG1Ring, 0) : 0;
  }
  const bool ox = x >= bx.lo[0] && x < bx.hi[0] && y >= bx.lo[1] && y < bx.hi[1];
  const bool oy = x >= by.lo[0] && x < by.hi[0] && y >= by.lo[1] && y < by.hi[1];
  const bool oz = x >= bz.lo[0] && x < bz.hi[0] && y >= bz.lo[1] && y < bz.hi[1];
  const int e = (ty + kG1Ring) * kG1SX + tx + kG1Ring;  // this column's cell in the plane tile
  // loads run ahead of their use: the column's z+3 and the ring's plane z+2 are requested while
  // plane z is formed, so no step waits on a load issued in the same step
  R w[FPB][7], rv[FPB][2][3];
  long long oc = pcol + (long long)(zs - 3) * sz;  // column offset of the next load
  long long orr = (long long)zs * sz;              // ring offset (plus r_p) of the next load
#pragma unroll
  for (int q = 0; q < FPB; ++q) {
#pragma unroll
    for (int k = 0; k < 6; ++k) w[q][k] = col ? src[q][oc + k * sz] : R(0);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      rv[q][h][0] = r_ok[h] ? src[q][r_p[h] + orr] : R(0);
      rv[q][h][1] = r_ok[h] ? src[q][r_p[h] + orr + sz] : R(0);
    }
  }
  oc += 6 * sz;
  orr += 2 * sz;
  long long p = pcol + (long long)zs * sz;
  for (int z = zs; z < ze; ++z, p += sz, oc += sz, orr += sz) {
    const int buf = (z - zs) & 1;
#pragma unroll
    for (int q = 0; q < FPB; ++q) {
      w[q][6] = col ? src[q][oc] : R(0);
#pragma unroll
      for (int h = 0; h < 2; ++h) rv[q][h][2] = r_ok[h] ? src[q][r_p[h] + orr] : R(0);
      R* pl = plane[buf][q];
      pl[e] = w[q][3];
#pragma unroll
      for (int h = 0; h < 2; ++h)
        if (r_off[h] >= 0) pl[r_off[h]] = rv[q][h][0];
    }
    __syncthreads();
    const bool zx = ox && z >= bx.lo[2] && z < bx.hi[2];
    const bool zy = oy && z >= by.lo[2] && z < by.hi[2];
    const bool zz = oz && z >= bz.lo[2] && z < bz.hi[2];
#pragma unroll
    for (int q = 0; q < FPB; ++q) {
      const R* pl = plane[buf][q];
      if (zx) A.g1[0][fo[q] + p] = stencil_E6x60(pl + e, 0, 1);
      if (zy) A.g1[1][fo[q] + p] = stencil_E6x60(pl + e, 0, kG1SX);
      if (zz) A.g1[2][fo[q] + p] = stencil_E6x60(w[q], 3, 1);
#pragma unroll
      for (int k = 0; k < 6; ++k) w[q][k] = w[q][k + 1];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        rv[q][h][0] = rv[q][h][1];
        rv[q][h][1] = rv[q][h][2];
      }
    }
  }
}

// The same derivatives (FP32) with four consecutive x-cells per thread, for layouts whose padded rows
// are 16-byte aligned: a block of 8 x 16 threads owns a 32 x 16 tile of columns, keeps the seven
// planes z-3 .. z+3 of its four cells as float4 registers (plus the next GBR_G1V_AHEAD planes in
// flight), and puts each plane with a ring of one float4 column and three rows around the tile into
// shared memory.  An x-derivative of four cells then takes two 16-byte shared loads, a y-derivative
// six, and the stores go out as float4 where the four cells lie in the box.  The arithmetic per cell
// is stencil_E6x60's, so every output equals k_grad1t's and body_grad1's.  128^3 mixed TGV: 0.066
// against 0.075 ms per launch (39 M against 62 M warp instructions; 24 warps per SM, latency- and
// barrier-stalled at 54 % issue, DRAM at 39 %).  Measured and not kept: one plane ahead (89
// registers, 5 blocks per SM; +0.4 % per step) or three, 8 blocks per SM (64 registers), the z loop
// unrolled over a register ring (no queue moves; +0.7 %), and the planes brought in by TMA into a
// ring of nine shared slots with mbarriers (no registers for planes in flight, but 15 shared loads
// per plane instead of 8: 45 M warp instructions, +0.3 %).
constexpr int kGVX = 8, kGVY = 16;                // threads along x (four cells each) and y
constexpr int kGVW = kGVX + 2, kGVR = kGVY + 6;   // float4 columns and rows of a plane tile
constexpr int kGVHalo = 6 * kGVW + 2 * kGVY;      // 92 ring float4s per plane
#ifndef GBR_G1V_BLOCKS
#define GBR_G1V_BLOCKS 24                         // blocks per SM the z-chunks aim at
#endif
#ifndef GBR_G1V_AHEAD
#define GBR_G1V_AHEAD 2                           // planes of loads in flight
#endif
#ifndef GBR_G1V_MINB
#define GBR_G1V_MINB 6                            // launch bound: blocks per SM
#endif

__device__ __forceinline__ float4 g1v_ld(const float* p, bool ok) {
  return ok ? *reinterpret_cast<const float4*>(p) : make_float4(0.f, 0.f, 0.f, 0.f);
}
__device__ __forceinline__ float g1v_c(const float4& v, int m) {
  return m == 0 ? v.x : m == 1 ? v.y : m == 2 ? v.z : v.w;
}
// stencil_E6x60 of the 7 values a[m .. m + 6] of the 10 cells x - 3 .. x + 6 around a thread's four
// cells x .. x + 3
__device__ __forceinline__ float g1v_e6(const float* a, int m) { return stencil_E6x60(a + m, 3, 1); }

// One block's tile t (tile in x, tile in y, chunk of planes; x fastest) of field f, through the
// block's double-buffered plane tiles in shared memory.  A block may run several tiles in a row:
// the barrier on entry lets every thread finish reading the previous tile's last plane before the
// buffers are written again.
__device__ __forceinline__ void grad1v_tile(const RhsArgsT<float>& A, const Box& U, const Box& bx, const Box& by,
                                            const Box& bz, int tiles_x, int tiles_y, int zchunk, int t, int f,
                                            float4 (*plane)[kGVR * kGVW]) {
  constexpr int NV = 5;
  __syncthreads();
  const Layout& L = A.L;
  const int tid = threadIdx.x, tx = tid % kGVX, ty = tid / kGVX;
  const int tlx = t % tiles_x, tly = (t / tiles_x) % tiles_y, chunk = t / (tiles_x * tiles_y);
  // the tile's first cell: x on a 16-byte boundary of the padded row (x + hp a multiple of 4)
  const int x0 = -L.hp[0] + tlx * 4 * kGVX, y0 = U.lo[1] + tly * kGVY;
  const int x = x0 + 4 * tx, y = y0 + ty;
  const int zs = U.lo[2] + chunk * zchunk, ze = min(zs + zchunk, U.hi[2]);
  const long long PC = L.pcount, sz = L.ps[2];
  const float* src = (f < NV) ? A.prim + f * PC : A.temp;
  const long long fo = f * PC;
  // a float4 of cells xq .. xq + 3 of row y is read where it lies in the padded box (outside it no
  // output needs it); along z the planes read, zs - 3 .. ze + 2, lie in the padded range
  auto inside = [&](int xq, int cy) {
    return xq >= -L.hp[0] && xq + 4 <= L.n[0] + L.hp[0] && cy >= -L.hp[1] && cy < L.n[1] + L.hp[1];
  };
  const bool col = inside(x, y);
  const long long pcol = col ? pidx(L, x, y, 0) : 0;
  // the ring float4 this thread loads (threads 0 .. 91): its slot and padded offset
  int h_slot = -1;
  bool h_ok = false;
  long long h_p = 0;
  if (tid < kGVHalo) {
    int r, c;
    if (tid < 3 * kGVW) {
      r = tid / kGVW;
      c = tid % kGVW;
    } else if (tid < 3 * kGVW + 2 * kGVY) {
      const int q = tid - 3 * kGVW;
      r = 3 + q / 2;
      c = (q % 2) ? kGVW - 1 : 0;
    } else {
      const int q = tid - 3 * kGVW - 2 * kGVY;
      r = 3 + kGVY + q / kGVW;
      c = q % kGVW;
    }
    h_slot = r * kGVW + c;
    const int xq = x0 - 4 + 4 * c, cy = y0 - 3 + r;
    h_ok = inside(xq, cy);
    h_p = h_ok ? pidx(L, xq, cy, 0) : 0;
  }
  const int e = (ty + 3) * kGVW + tx + 1;  // this thread's float4 in the plane tile
  // the (x, y) tests of this thread's four cells against the three boxes
  auto inb = [&](const Box& b, int m) { return x + m >= b.lo[0] && x + m < b.hi[0] && y >= b.lo[1] && y < b.hi[1]; };
  bool in[3][4];
  #pragma unroll
  for (int m = 0; m < 4; ++m) {
    in[0][m] = inb(bx, m);
    in[1][m] = inb(by, m);
    in[2][m] = inb(bz, m);
  }
  // the planes z - 3 .. z + 3 of the column and, in flight, the next AH; the ring's plane z and the
  // next AH (a plane is read only up to ze + 2, the ring's only below ze).  (The z loop unrolled over
  // a register ring, so that no value moves, measured slower.)
  constexpr int AH = GBR_G1V_AHEAD;
  float4 w[7 + AH], hv[1 + AH];
  #pragma unroll
  for (int kq = 0; kq < 6 + AH; ++kq) w[kq] = g1v_ld(src + pcol + (long long)(zs - 3 + kq) * sz, col && zs - 3 + kq <= ze + 2);
  #pragma unroll
  for (int kq = 0; kq < AH; ++kq) hv[kq] = g1v_ld(src + h_p + (long long)(zs + kq) * sz, h_ok && zs + kq < ze);
  long long p = pcol + (long long)zs * sz;
  for (int z = zs; z < ze; ++z, p += sz) {
    const int buf = (z - zs) & 1;
    // the loads of the plane AH ahead, in flight while this plane is formed
    w[6 + AH] = g1v_ld(src + p + (3 + AH) * sz, col && z + 3 + AH <= ze + 2);
    hv[AH] = g1v_ld(src + h_p + (long long)(z + AH) * sz, h_ok && z + AH < ze);
    plane[buf][e] = w[3];
    if (h_slot >= 0) plane[buf][h_slot] = hv[0];
    __syncthreads();
    const float4* pl = plane[buf];
    const bool zx = z >= bx.lo[2] && z < bx.hi[2], zy = z >= by.lo[2] && z < by.hi[2], zz = z >= bz.lo[2] && z < bz.hi[2];
    float4 o[3];
    {
      const float4 l = pl[e - 1], r = pl[e + 1];
      const float a[10] = {l.y, l.z, l.w, w[3].x, w[3].y, w[3].z, w[3].w, r.x, r.y, r.z};
      o[0] = make_float4(g1v_e6(a, 0), g1v_e6(a, 1), g1v_e6(a, 2), g1v_e6(a, 3));
    }
    {
      const float4 m3 = pl[e - 3 * kGVW], m2 = pl[e - 2 * kGVW], m1 = pl[e - kGVW];
      const float4 p1 = pl[e + kGVW], p2 = pl[e + 2 * kGVW], p3 = pl[e + 3 * kGVW];
      float v[4];
      #pragma unroll
      for (int m = 0; m < 4; ++m) {
        const float c7[7] = {g1v_c(m3, m), g1v_c(m2, m), g1v_c(m1, m), g1v_c(w[3], m), g1v_c(p1, m), g1v_c(p2, m), g1v_c(p3, m)};
        v[m] = stencil_E6x60(c7, 3, 1);
      }
      o[1] = make_float4(v[0], v[1], v[2], v[3]);
    }
    {
      float v[4];
      #pragma unroll
      for (int m = 0; m < 4; ++m) {
        const float c7[7] = {g1v_c(w[0], m), g1v_c(w[1], m), g1v_c(w[2], m), g1v_c(w[3], m), g1v_c(w[4], m), g1v_c(w[5], m), g1v_c(w[6], m)};
        v[m] = stencil_E6x60(c7, 3, 1);
      }
      o[2] = make_float4(v[0], v[1], v[2], v[3]);
    }
    const bool zd[3] = {zx, zy, zz};
    #pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (!zd[d]) continue;
      float* out = A.g1[d] + fo + p;
      if (in[d][0] && in[d][1] && in[d][2] && in[d][3]) {
        *reinterpret_cast<float4*>(out) = o[d];
      } else {
        #pragma unroll
        for (int m = 0; m < 4; ++m)
          if (in[d][m]) out[m] = g1v_c(o[d], m);
      }
    }
    #pragma unroll
    for (int kq = 0; kq < 6 + AH; ++kq) w[kq] = w[kq + 1];
    #pragma unroll
    for (int kq = 0; kq < AH; ++kq) hv[kq] = hv[kq + 1];
  }
}

__global__ void __launch_bounds__(kGVX * kGVY, GBR_G1V_MINB) k_grad1v(RhsArgsT<float> A, Box U, Box bx, Box by, Box bz, int tiles_x,
                                                      int tiles_y, int zchunk) {
  __shared__ float4 plane[2][kGVR * kGVW];
  grad1v_tile(A, U, bx, by, bz, tiles_x, tiles_y, zchunk, (int)blockIdx.x, (int)blockIdx.y, plane);
}

// MIG4: one thread per (line, field); blockIdx.y is the field (primitives, then T)
template <int ND, class R = double>
__global__ void k_ig4(RhsArgsT<R> A, int e, Box lines, const R* table) {
  constexpr int NV = ND + 2;
  BOX_THREAD(lines);
  const int f = blockIdx.y;
  const long long PC = A.L.pcount;
  const R* src = (f < NV) ? A.prim + f * PC : A.temp;
  ig4_line(A.L, table, e, src, A.g1[e] + f * PC, i, j, k);
}

__global__ void k_ig4_factor(double* table, int n, int periodic) { ig4_factor(table, n, periodic != 0); }

// one element from global into shared memory without a register round trip (cp.async)
template <class R>
__device__ __forceinline__ void cp_async_elem(R* dst, const R* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(__cvta_generic_to_global(src)),
               "n"((int)sizeof(R))
               : "memory");
}

// MIG4 with the lines staged in shared memory: a block of kIg4Lines threads takes kIg4Lines
// neighbouring lines of one field (neighbours along axis a: x for y- and z-lines, y for
// x-lines), loads their padded rows with coalesced asynchronous copies (consecutive threads read
// consecutive addresses: along the line for x-lines, across the lines otherwise; all of a tile's
// copies are in flight together, where loads through registers left the kernel waiting on a few
// at a time), solves each line in its own thread from shared memory (in place; rows of odd
// length, so the threads' accesses fall in distinct banks), and stores the derivative rows back
// with coalesced writes.  The x-lines, which a thread per line in global memory walks with a
// stride across the warp, become coalesced.  The y- and z-lines take the TMA form below where
// its alignment rules hold.
constexpr int kIg4Lines = 32;
// The FP32 solves read the factor table from shared memory (a uniform load per row that no longer
// waits on L1); the FP64 solves, bound by the FP64 pipe, keep it in global memory, where it costs
// no shared memory and so no resident blocks.
template <class R>
constexpr bool kIg4StageTable = sizeof(R) == sizeof(float);

template <int ND, class R>
__global__ void __launch_bounds__(kIg4Lines) k_ig4s(RhsArgsT<R> A, int e, Box lines, const R* table,
                                                      int srow, int tlen) {
  constexpr int NV = ND + 2;
  extern __shared__ __align__(16) unsigned char ig4_smem[];
  R* F = reinterpret_cast<R*>(ig4_smem);
  const Layout& L = A.L;
  // (e, a, b) is (x, y, z), (y, x, z) or (z, x, y): selects, no arrays indexed at run time
  const bool ex = (e == 0), ey = (e == 1);
  const int n = ex ? L.n[0] : (ey ? L.n[1] : L.n[2]), M = n + 2 * H;
  const int loa = ex ? lines.lo[1] : lines.lo[0], na = (ex ? lines.hi[1] : lines.hi[0]) - loa;
  const int lob = (ex || ey) ? lines.lo[2] : lines.lo[1];
  const int tiles = (na + kIg4Lines - 1) / kIg4Lines;
  const int ta = blockIdx.x % tiles, tb = blockIdx.x / tiles;
  const int nl = min(kIg4Lines, na - ta * kIg4Lines);
  const int ca = loa + ta * kIg4Lines, cb = lob + tb;
  // padded cell -H of the tile's first line
  const long long base = ex ? pidx(L, -H, ca, cb) : (ey ? pidx(L, ca, -H, cb) : pidx(L, ca, cb, -H));
  const long long sa = ex ? L.ps[1] : 1, se = ex ? 1 : (ey ? L.ps[1] : L.ps[2]);
  const int f = blockIdx.y;
  const long long PC = L.pcount;
  const R* src = (f < NV) ? A.prim + f * PC : A.temp;
  R* dst = (ex ? A.g1[0] : (ey ? A.g1[1] : A.g1[2])) + f * PC;
  const bool per = ex ? L.per[0] != 0 : (ey ? L.per[1] != 0 : L.per[2] != 0);
  const int tid = threadIdx.x;
  // FP32: the factor table staged beside the rows (every line reads the same entry at each row)
  const R* T = table;
  if constexpr (kIg4StageTable<R>) {
    R* Ts = F + kIg4Lines * srow;
    for (int i = tid; i < tlen; i += kIg4Lines) Ts[i] = table[i];
    T = Ts;
  }
  // asynchronous element copies (cp.async): every load of the tile is in flight at once
  if (ex) {
    for (int l = 0; l < nl; ++l)
      for (int m = tid; m < M; m += kIg4Lines) cp_async_elem(F + l * srow + m, src + base + l * sa + m);
  } else if (tid < nl) {
    for (int m = 0; m < M; ++m) cp_async_elem(F + tid * srow + m, src + base + tid + m * se);
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  if (tid < nl) ig4_solve(T, n, per, F + tid * srow + H, F + tid * srow + H, 1, F + tid * srow, 1);
  __syncthreads();
  // rows written by the solve: the n cells and 3 images each side (periodic), the padded line (open)
  const int m0 = per ? H - 3 : 0, m1 = per ? H + n + 3 : M;
  if (ex) {
    for (int l = 0; l < nl; ++l)
      for (int m = m0 + tid; m < m1; m += kIg4Lines) dst[base + l * sa + m] = F[l * srow + m];
  } else if (tid < nl) {
    for (int m = m0; m < m1; ++m) dst[base + tid + m * se] = F[tid * srow + m];
  }
}

// shared-memory row length (odd) and bytes of the staged MIG4 kernel for a line of n cells
inline int ig4_srow(int n) { return (n + 2 * H) | 1; }
template <class R>
size_t ig4_smem_bytes(int n, bool per) {
  return sizeof(R) * ((size_t)kIg4Lines * ig4_srow(n) + (kIg4StageTable<R> ? (size_t)ig4_table_len(n, per) : 0));
}
constexpr size_t kIg4SmemMax = 200 * 1024;

// The same solves with the tile brought in by one TMA bulk copy (cp.async.bulk.tensor): for y- and
// z-lines the 32 neighbouring lines are the box {32 along x, the padded line along e} of the field,
// a single asynchronous copy into shared memory (laid out [point][line]: the per-thread solve reads
// consecutive words, no bank conflicts) completed on an mbarrier.  Tiles start at a padded x that is
// a multiple of 4, so the copy's innermost coordinate is 16-byte aligned; the host uses this form
// only when the row pitch is a multiple of 16 bytes and the padded line fits one box (<= 256).  The
// wait is bounded: if the copy has not completed after kTmaSpin try_wait polls (each suspending
// for at most about kTmaWaitNs), the block flags it in err[1] (gbr_sync reports a timeout), waits
// once more, boundedly, for the copy to land, and leaves without writing its derivatives.
constexpr int kTmaSpin = 1 << 16;
constexpr unsigned kTmaWaitNs = 1000;  // suspend-time hint of one try_wait, ns
template <class R>
size_t ig4t_smem_bytes(int n, bool per) {
  return sizeof(R) * ((size_t)kIg4Lines * (n + 2 * H) + (kIg4StageTable<R> ? (size_t)ig4_table_len(n, per) : 0)) + 128;
}

// bounded wait on phase 0 of the block's mbarrier: true once the copy has landed
__device__ __forceinline__ bool tma_wait(unsigned bar, int spins) {
  unsigned done = 0;
  for (int it = 0; it < spins && !done; ++it)
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0, %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(bar), "r"(kTmaWaitNs)
        : "memory");
  return done != 0;
}

// The timeout path of the bounded wait, run on purpose: one block waits on an mbarrier that
// expects an arrival nobody makes (no copy is issued, so nothing is in flight when it leaves) and
// flags err[1] as a line-solve block whose tile never landed would.
__global__ void k_wait_check(int polls, int* err) {
  __shared__ __align__(8) unsigned long long mbar;
  const unsigned bar = (unsigned)__cvta_generic_to_shared(&mbar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (!tma_wait(bar, polls) && threadIdx.x == 0) atomicOr(err + 1, 1);
}

template <int ND, class R>
__global__ void __launch_bounds__(kIg4Lines) k_ig4t(RhsArgsT<R> A, int e, Box lines, const R* table, int tlen, int x0p,
                                                     const __grid_constant__ CUtensorMap tm_prim,
                                                     const __grid_constant__ CUtensorMap tm_temp, int* err) {
  constexpr int NV = ND + 2;
  extern __shared__ __align__(16) unsigned char ig4t_smem[];
  __shared__ __align__(8) unsigned long long mbar;
  // the copy's destination on a 128-byte boundary (the allocation carries 128 bytes of slack)
  const unsigned s0 = (unsigned)__cvta_generic_to_shared(ig4t_smem);
  const unsigned pad = (128u - (s0 & 127u)) & 127u;
  R* F = reinterpret_cast<R*>(ig4t_smem + pad);
  const unsigned dst = s0 + pad;
  const Layout& L = A.L;
  const int n = (e == 1) ? L.n[1] : L.n[2], M = n + 2 * H;
  // the third axis b (extent 1 in 2D): z for y-lines, y for z-lines (selects, no indexed arrays)
  const bool ey = (e == 1);
  const int lob = ey ? lines.lo[2] : lines.lo[1], hpb = ey ? L.hp[2] : L.hp[1];
  const int tiles = (lines.hi[0] + L.hp[0] - x0p + kIg4Lines - 1) / kIg4Lines;
  const int tx = blockIdx.x % tiles, tb = blockIdx.x / tiles;
  const int xs = x0p + tx * kIg4Lines;  // padded x of the tile's first line (a multiple of 4)
  const int cb = lob + tb + hpb;        // padded coordinate of the tile along b
  const int f = blockIdx.y;
  const int tid = threadIdx.x;
  const unsigned bar = (unsigned)__cvta_generic_to_shared(&mbar);
  const unsigned bytes = (unsigned)(sizeof(R) * kIg4Lines * M);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    const int c1 = ey ? 0 : cb, c2 = ey ? cb : 0;  // the line starts at padded 0 along e
    if (f < NV)
      asm volatile(
          "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
          "[%6];" ::"r"(dst),
          "l"(reinterpret_cast<unsigned long long>(&tm_prim)), "r"(xs), "r"(c1), "r"(c2), "r"(f), "r"(bar)
          : "memory");
    else
      asm volatile(
          "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
          "[%5];" ::"r"(dst),
          "l"(reinterpret_cast<unsigned long long>(&tm_temp)), "r"(xs), "r"(c1), "r"(c2), "r"(bar)
          : "memory");
  }
  const R* T = table;
  if constexpr (kIg4StageTable<R>) {  // FP32: the factor table, staged while the tile is in flight
    R* Ts = F + kIg4Lines * M;
    for (int i = tid; i < tlen; i += kIg4Lines) Ts[i] = table[i];
    T = Ts;
    __syncwarp();
  }
  if (!tma_wait(bar, kTmaSpin)) {
    // the copy did not land in time: flag it, give the copy a last bounded chance to finish before
    // the block's shared memory is released, and leave the derivatives of this tile unwritten
    if (tid == 0) atomicOr(err + 1, 1);
    tma_wait(bar, kTmaSpin);
    return;
  }
  // this thread's line: cell x = xs - hp0 + tid, solved and stored when it lies in the lines box
  const int cx = xs - L.hp[0] + tid;
  if (cx < lines.lo[0] || cx >= lines.hi[0]) return;
  const bool per = ey ? L.per[1] != 0 : L.per[2] != 0;
  const int cl = lob + tb;
  const long long base = ey ? pidx(L, cx, -H, cl) : pidx(L, cx, cl, -H);  // padded cell -H of this thread's line
  const long long se = ey ? L.ps[1] : L.ps[2];
  R* out = (ey ? A.g1[1] : A.g1[2]) + f * L.pcount + base;
  // forward sweep in the shared column, backward sweep stored straight to the derivative (the
  // threads of the warp write neighbouring x: coalesced): the n cells and 3 images each side
  // (periodic), the padded line (open)
  R* col = F + tid + H * kIg4Lines;
  ig4_solve(T, n, per, col, col, kIg4Lines, out, se);
}

template <int ND, class R = double>
__global__ void k_grad2(RhsArgsT<R> A, Box b0, Box b1, Box b2) {
  GRAD_THREAD(b0, b1, b2);
  body_grad2<ND>(A, e, i, j, k);
}

// Interfaces whose App. E test failed, handed from their thread to a worker thread of the block.
template <int ND, class R>
struct BoundSlot {
  FaceIx<R> p1;
  unsigned limit;
  R nu[ND];
  R ra, a2;
  R Wd[3][ND + 2];
  R dL[ND + 2], dR[ND + 2];
};

// One interface per thread, with the limiter's bound work compacted over the block: the FP64
// pipe is charged per warp instruction, so bounds computed in the threads that need them cost
// every warp containing one such interface; here the interfaces that failed the test are queued
// in shared memory and the block's first threads compute all of their bounds (the same
// arithmetic per interface), then every thread finishes its own flux.  No thread leaves before
// the block's barriers.
template <int ND, bool VISC, bool MOV, class R, int DD = -1>
__device__ __forceinline__ void face_block(const RhsArgsT<R>& A, int d, bool valid, int i, int j, int k,
                                           BoundSlot<ND, R>* slots, int* count) {
  constexpr int NV = ND + 2;
  FaceCtx<ND, R> C;
  C.limit = 0;
  if (valid) face_unlimited<ND, MOV, R, DD>(A, d, i, j, k, C);
  if (threadIdx.x == 0) *count = 0;
  __syncthreads();
  int slot = -1;
  if (C.limit) {
    slot = atomicAdd(count, 1);
    BoundSlot<ND, R>& S = slots[slot];
    S.p1 = C.p1;
    S.limit = C.limit;
    S.ra = C.ra;
    S.a2 = C.a2;
    #pragma unroll
    for (int a = 0; a < ND; ++a) S.nu[a] = C.nu[a];
    #pragma unroll
    for (int c = 0; c < NV; ++c) {
      S.Wd[0][c] = C.Wd[0][c];
      S.Wd[1][c] = C.Wd[1][c];
      S.Wd[2][c] = C.Wd[2][c];
      S.dL[c] = C.dL[c];
      S.dR[c] = C.dR[c];
    }
  }
  __syncthreads();
  const int n = *count;
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    BoundSlot<ND, R>& S = slots[t];
    face_bounds<ND, R, DD>(A, d, S.nu, S.ra, S.a2, S.p1, S.limit, S.Wd, S.dL, S.dR);
  }
  __syncthreads();
  if (slot >= 0) {
    #pragma unroll
    for (int c = 0; c < NV; ++c) {
      C.dL[c] = slots[slot].dL[c];
      C.dR[c] = slots[slot].dR[c];
    }
  }
  if (valid) face_flux<ND, VISC, MOV, R, DD>(A, d, i, j, k, C);
}

// Bound work compacted over the block in both precisions (FP64: FP64-pipe bound, -7 % on the
// 128^3 TGV; FP32, where the bounds form the four cells' f'': -5 % against one interface per thread)
template <int DD>
__host__ __device__ constexpr int face_bs() { return DD == 0 ? GBR_FACE_BLOCK_X : GBR_FACE_BLOCK; }
template <class R, int DD>
__host__ __device__ constexpr int face_mb() {
  return sizeof(R) == 4 ? (DD == 0 ? GBR_FACE_MIN_BLOCKS_F32_X : GBR_FACE_MIN_BLOCKS_F32)
                        : (DD == 0 ? GBR_FACE_MIN_BLOCKS_X : GBR_FACE_MIN_BLOCKS);
}
template <class R, int ND, int DD>
__host__ __device__ constexpr int face_xt() {
  return (ND == 3 && DD == 0) ? (sizeof(R) == 4 ? GBR_FACE_XT_WX_F32 : GBR_FACE_XT_WX) : 0;
}

// The transposed x-sweep mapping (WX > 0, blocks of BS threads): a warp holds WX consecutive
// x-interfaces of 32 / WX consecutive x-lines, the lines (j, k) numbered j fastest so that only the
// box's last line group is ragged.  Blocks of a box, and the interface of thread `tid` of block `blk`
// (false past the box).  int: the lines of a face box are below its interfaces, which the 32-bit
// offset check keeps below 2^32 / 9.
__host__ __device__ inline long long face_xt_blocks(const Box& b, int bs, int wx) {
  const int BX = wx * (bs / 32), BY = 32 / wx;
  const long long nx = b.hi[0] - b.lo[0], nl = (long long)(b.hi[1] - b.lo[1]) * (b.hi[2] - b.lo[2]);
  return ((nx + BX - 1) / BX) * ((nl + BY - 1) / BY);
}
template <int BS, int WX>
__device__ __forceinline__ bool face_xt_coord(const Box& b, int blk, int tid, int& i, int& j, int& k) {
  constexpr int BX = WX * (BS / 32), BY = 32 / WX;
  const int nx = b.hi[0] - b.lo[0], ny = b.hi[1] - b.lo[1], nl = ny * (b.hi[2] - b.lo[2]);
  const int gx = (nx + BX - 1) / BX, lane = tid % 32;
  const int line = (blk / gx) * BY + lane / WX;
  i = b.lo[0] + (blk % gx) * BX + (tid / 32) * WX + lane % WX;
  j = b.lo[1] + line % ny;
  k = b.lo[2] + line / ny;
  return i < b.hi[0] && line < nl;
}

template <int ND, bool VISC, bool MOV, class R = double, int DD = -1>
__global__ void __launch_bounds__(face_bs<DD>(), face_mb<R, DD>())
    k_face(RhsArgsT<R> A, int d, Box b) {
  constexpr int BS = face_bs<DD>();
  __shared__ BoundSlot<ND, R> slots[BS];
  __shared__ int count;
  bool valid;
  int i = 0, j = 0, k = 0;
  if constexpr (face_xt<R, ND, DD>() > 0) {
    valid = face_xt_coord<BS, face_xt<R, ND, DD>()>(b, (int)blockIdx.x, (int)threadIdx.x, i, j, k);
  } else {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    valid = t < box_size(b);
    if (valid) box_coord(b, t, i, j, k);
  }
  face_block<ND, VISC, MOV, R, DD>(A, d, valid, i, j, k, slots, &count);
}

template <int ND, bool MOV, class R = double, bool SP = true>
__global__ void __launch_bounds__(kBlock, kStreamBlocks) k_update(UpdArgsT<R> U, Box b, int* err) {
  BOX_THREAD(b);
  if (body_update<ND, MOV, R, SP>(U, i, j, k)) atomicOr(err, 1);
}

__global__ void k_dt_f32(DtArgs D, float* mh32, float* mt32, float* jac32, Box b) {
  BOX_THREAD(b);
  body_dt_f32(D, mh32, mt32, jac32, i, j, k);
}

template <int ND, class R = double, bool GS = false>
__global__ void k_dt(DtArgs D, Box b, unsigned long long* minbits) {
  // the minimum is taken in the path's type (exact: conversion to FP64 is monotone and exact),
  // and converted once per block -- on the mixed path no FP64-pipe work per cell but the state's
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  R v = R(HUGE_VAL);
  if (t < box_size(b)) {
    int i, j, k;
    box_coord(b, t, i, j, k);
    v = body_dt_r<ND, R, GS>(D, i, j, k);
  }
  // fmin (fminf for FP32, on the ALU pipe) passes over a NaN of a broken state as before
  for (int off = 16; off > 0; off >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, off));
  __shared__ R wmin[kBlock / 32];
  if ((threadIdx.x & 31) == 0) wmin[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    R w = (threadIdx.x < blockDim.x / 32) ? wmin[threadIdx.x] : R(HUGE_VAL);
    for (int off = 16; off > 0; off >>= 1) w = fmin(w, __shfl_xor_sync(0xffffffffu, w, off));
    // positive doubles order like their bit patterns
    if (threadIdx.x == 0) atomicMin(minbits, (unsigned long long)__double_as_longlong(fmin(1.0e300, double(w))));
  }
}

__global__ void k_dt_init(unsigned long long* minbits) { *minbits = (unsigned long long)__double_as_longlong(1.0e300); }

__global__ void k_dt_final(double* scal, const unsigned long long* minbits, double cfl) {
  scal[S_DT] = cfl * __longlong_as_double((long long)*minbits);
}

__global__ void k_set_scalar(double* scal, int idx, double v) { scal[idx] = v; }
__global__ void k_to_f32(const double* src, float* dst, long long n) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) dst[t] = (float)src[t];
}
__global__ void k_advance_time(double* scal) { scal[S_T] += scal[S_DT]; }

// ---------------------------------------------------------------------------
// workspace plan
// ---------------------------------------------------------------------------
struct Plan {
  size_t off[64];
  size_t len[64];
  int count = 0;
  size_t total = 0;
  int add(size_t bytes) {
    total = (total + 255) & ~(size_t)255;
    off[count] = total;
    len[count] = bytes;
    total += bytes;
    return count++;
  }
};

enum Slot {
  SL_Q0, SL_Q1, SL_Q2, SL_PRIM, SL_TEMP, SL_G1, SL_G2, SL_FLUX, SL_NODES, SL_NVEL, SL_XC, SL_VC, SL_XD, SL_MH,
  SL_DET, SL_MU, SL_MT, SL_FH, SL_FU, SL_FT, SL_GCL, SL_JAC, SL_SIGMA, SL_INFLOW, SL_SCAL, SL_ERR, SL_IG4, SL_FH32, SL_FU32,
  SL_FT32, SL_IG4F, SL_MH32, SL_MT32, SL_JAC32, SL_GEOT, SL_GEOW, SL_FG, SL_GDT, SL_COUNT
};

struct Sizes {
  size_t bytes[SL_COUNT];
};

Layout layout_of(const gbr_params* p);

constexpr int kMaxAxisCells = 1 << 24;  // cells along one axis
constexpr int kMaxGhostNodes = 1024;    // node layers beyond a non-periodic side

bool valid_params(const gbr_params* p, std::string& why) {
  if (!p) { why = "null params"; return false; }
  if (p->ndim != 2 && p->ndim != 3) { why = "ndim must be 2 or 3"; return false; }
  // bounds before any size arithmetic: padded extents n + 2 * (6 + 10) and node counts stay far inside int
  if (p->ghost_nodes < 0 || p->ghost_nodes > kMaxGhostNodes) { why = "ghost_nodes out of range"; return false; }
  for (int d = 0; d < p->ndim; ++d) {
    if (p->n[d] < 1) { why = "empty axis"; return false; }
    if (p->n[d] > kMaxAxisCells) { why = "axis too long"; return false; }
    if (p->periodic[d] && p->n[d] < H) { why = "a periodic axis needs at least 6 cells"; return false; }
    if (!p->periodic[d] && p->ghost_nodes != 0 && p->ghost_nodes < E) {
      why = "a non-periodic axis needs ghost_nodes >= 10, or 0 (walls, App. C metrics)";
      return false;
    }
    if (!p->periodic[d] && p->ghost_nodes == 0 && p->n[d] < 2 * H) {
      why = "an axis without ghost nodes needs at least 12 cells";
      return false;
    }
    if (!p->periodic[d]) {
      for (int s = 0; s < 2; ++s) {
        int bc = p->bc[d][s];
        if (bc != GBR_BC_ZEROGRAD && bc != GBR_BC_INFLOW && bc != GBR_BC_WALL) {
          why = "unknown boundary condition";
          return false;
        }
        if (bc == GBR_BC_INFLOW && !(d == 0 && s == 0)) { why = "inflow is supported on the x-low side only"; return false; }
        if (bc == GBR_BC_WALL && p->n[d] < H) { why = "a wall axis needs at least 6 cells"; return false; }
      }
    }
  }
  if (!(p->gamma > 1.0)) { why = "gamma must exceed 1"; return false; }
  if (p->reynolds > 0.0 && !(p->prandtl > 0.0)) { why = "prandtl must be positive"; return false; }
  if (p->sutherland_s > 0.0 && !(p->t_ref > 0.0)) { why = "t_ref must be positive"; return false; }
  if (p->precision != GBR_PREC_FP64 && p->precision != GBR_PREC_MIXED) { why = "unknown precision"; return false; }
  for (int d = 0; d < p->ndim; ++d)
    if (!p->periodic[d] && p->ghost_nodes == 0 && p->moving) {
      why = "moving meshes need ghost nodes on non-periodic axes";
      return false;
    }
  if (p->gradient_scheme != GBR_GRAD_MEG6 && p->gradient_scheme != GBR_GRAD_MIG4) {
    why = "unknown gradient scheme";
    return false;
  }
  for (int d = 0; d < p->ndim; ++d)
    if (p->gradient_scheme == GBR_GRAD_MIG4 && p->n[d] < 4) { why = "MIG4 needs at least 4 cells per axis"; return false; }
  long long cells = (long long)p->n[0] * p->n[1] * (p->ndim == 3 ? p->n[2] : 1);
  if (cells > (1LL << 34)) { why = "grid too large"; return false; }
  // the interface kernels address their arrays with 32-bit offsets: (fields + 1) x padded cells
  // and 9 x interfaces of a direction stay below 2^32 (a larger grid would not fit in memory)
  const Layout L = layout_of(p);
  long long fmax = 0;
  for (int d = 0; d < L.nd; ++d) fmax = std::max(fmax, L.fcount[d]);
  if ((long long)(L.nv + 1) * L.pcount >= (1LL << 32) || 9LL * fmax >= (1LL << 32) || L.ecount >= (1LL << 32) ||
      L.ncount >= (1LL << 32)) {
    why = "grid too large (32-bit array offsets)";
    return false;
  }
  return true;
}

Layout layout_of(const gbr_params* p) {
  int n[3] = {p->n[0], p->n[1], p->ndim == 3 ? p->n[2] : 1};
  int closed[3];
  for (int d = 0; d < 3; ++d) closed[d] = (d < p->ndim && !p->periodic[d] && p->ghost_nodes == 0) ? 1 : 0;
  int ig4_geo[3];
  for (int d = 0; d < 3; ++d) ig4_geo[d] = p->gradient_scheme == GBR_GRAD_MIG4 ? 1 : 0;
  return make_layout(p->ndim, n, p->periodic, closed, ig4_geo);
}

// bytes of one element of the arrays computed in the path's type
size_t elem_r(const gbr_params* p) { return p->precision == GBR_PREC_MIXED ? sizeof(float) : sizeof(double); }

Plan plan_of(const gbr_params* p, const Layout& L) {
  Plan P;
  const size_t D = sizeof(double);
  const int nv = L.nv, nd = L.nd;
  const bool visc = p->reynolds > 0.0;
  const bool mov = p->moving != 0;
  size_t fsum = 0;
  for (int d = 0; d < nd; ++d) fsum += (size_t)L.fcount[d];
  P.add(D * nv * L.ncells);                       // SL_Q0
  P.add(D * nv * L.ncells);                       // SL_Q1
  P.add(D * nv * L.ncells);                       // SL_Q2
  const size_t ER = elem_r(p);                    // primitives, gradients, fluxes: the path's type
  P.add(ER * nv * L.pcount);                      // SL_PRIM
  P.add(visc ? ER * L.pcount : 0);                // SL_TEMP
  P.add(ER * nd * (nv + (visc ? 1 : 0)) * L.pcount);  // SL_G1
  P.add(p->precision == GBR_PREC_MIXED ? 0 : ER * nd * nv * L.pcount);  // SL_G2 (FP64 path only)
  P.add(ER * nv * fsum);                          // SL_FLUX
  P.add(D * nd * L.ncount);                       // SL_NODES
  P.add(mov ? D * nd * L.ncount : 0);             // SL_NVEL
  P.add(D * nd * L.ecount);                       // SL_XC
  P.add(mov ? D * nd * L.ecount : 0);             // SL_VC
  P.add(D * 9 * L.ecount);                        // SL_XD
  P.add(D * 9 * L.ecount);                        // SL_MH
  P.add(D * L.ecount);                            // SL_DET
  P.add(visc ? D * 9 * L.ecount : 0);             // SL_MU
  P.add(mov ? D * 3 * L.ecount : 0);              // SL_MT
  P.add(D * nd * fsum);                           // SL_FH
  P.add(visc ? D * nd * nd * fsum : 0);           // SL_FU
  P.add(mov ? D * fsum : 0);                      // SL_FT
  P.add(mov ? D * L.ncells : 0);                  // SL_GCL
  P.add(D * L.ncells);                            // SL_JAC
  P.add(D * L.ncells);                            // SL_SIGMA
  P.add(D * nv * L.n[1] * L.n[2]);                // SL_INFLOW
  P.add(D * S_NSCAL);                             // SL_SCAL
  P.add(sizeof(int) * 4);                         // SL_ERR
  long long ig4 = 0;                               // SL_IG4: MIG4 line-solve factors per direction
  if (p->gradient_scheme == GBR_GRAD_MIG4)
    for (int d = 0; d < nd; ++d) ig4 += ig4_table_len(L.n[d], L.per[d] != 0);
  P.add(D * ig4);
  // mixed path: FP32 copies of the interface metrics the interface kernel reads
  const bool f32 = p->precision == GBR_PREC_MIXED;
  P.add(f32 ? sizeof(float) * nd * fsum : 0);                   // SL_FH32
  P.add(f32 && visc ? sizeof(float) * nd * nd * fsum : 0);      // SL_FU32
  P.add(f32 && mov ? sizeof(float) * fsum : 0);                 // SL_FT32
  P.add(f32 ? sizeof(float) * ig4 : 0);                         // SL_IG4F: FP32 copies of the MIG4 factors
  P.add(f32 ? sizeof(float) * 9 * L.ncells : 0);               // SL_MH32: the time step's cell metrics
  P.add(f32 && mov ? sizeof(float) * 3 * L.ncells : 0);        // SL_MT32
  P.add(f32 ? sizeof(float) * L.ncells : 0);                   // SL_JAC32
  // MIG4 metrics: Thomas factors of the extended and of the cell-metric lines per direction, and a
  // work array for the line solves
  const bool geo4 = p->gradient_scheme == GBR_GRAD_MIG4;
  long long geot = 0;
  if (geo4)
    for (int d = 0; d < nd; ++d) geot += 2LL * (L.n[d] + 2 * L.he[d]) + 2LL * (L.n[d] + 2 * L.cg[d]);
  P.add(D * geot);                                               // SL_GEOT
  P.add(geo4 ? D * L.ecount : 0);                                // SL_GEOW
  P.add(f32 ? 0 : D * fg_count(visc) * fsum);                    // SL_FG: FP64 interface geometry
  P.add(f32 || mov ? 0 : D * 2 * nd * L.ncells);                 // SL_GDT: FP64 time-step metric norms
  P.total = (P.total + 255) & ~(size_t)255;
  return P;
}

thread_local std::string g_global_error;

Box make_box(const Layout& L, const int lo[3], const int hi[3]) {
  Box b;
  for (int d = 0; d < 3; ++d) {
    if (d < L.nd) { b.lo[d] = lo[d]; b.hi[d] = hi[d]; }
    else { b.lo[d] = 0; b.hi[d] = 1; }
  }
  return b;
}

// box with per-axis pads: [lo_pad below 0, n + hi_pad)
Box pad_box(const Layout& L, int lo_pad, int hi_pad) {
  int lo[3], hi[3];
  for (int d = 0; d < 3; ++d) { lo[d] = -lo_pad; hi[d] = L.n[d] + hi_pad; }
  return make_box(L, lo, hi);
}

unsigned grid_of(const Box& b, int block) {
  long long n = box_size(b);
  return (unsigned)((n + block - 1) / block);
}

// blocks of one interface launch: one per block-size run of the box, or with the transposed
// x-sweep mapping one per (group of WX BS/32 x-interfaces, group of 32/WX x-lines)
template <class R, int ND, int DD>
unsigned face_grid(const Box& b) {
  constexpr int BS = face_bs<DD>();
  if constexpr (face_xt<R, ND, DD>() > 0) {
    return (unsigned)face_xt_blocks(b, BS, face_xt<R, ND, DD>());
  } else {
    return grid_of(b, BS);
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
struct gbr_ctx {
  gbr_params p;
  Layout L;
  Phys ph;
  cudaStream_t stream;
  char* ws;
  size_t ws_bytes;
  Plan plan;
  double* q[3];
  void *prim, *temp, *g1[3], *g2[3], *flux[3];  // element type double (FP64) or float (mixed)
  double *nodes, *nvel, *xc, *vc, *xd, *mh, *det, *mu, *mt, *fh[3], *fu[3], *ft[3], *gcl, *jac;
  double* fg[3];  // FP64 path: interface geometry derived from fh, fu (body_face_geo), or null
  double* gdt;    // FP64 path, static mesh: the time step's metric norms (body_dt_geo), or null
  float *fh32[3], *fu32[3], *ft32[3];  // mixed path: FP32 copies of the interface metrics
  float *mh32, *mt32, *jac32;          // mixed path: FP32 copies of the cell metrics (time step)
  double *sigma, *inflow, *scal;
  double* ig4[3];  // MIG4 line-solve factors per direction (or null)
  double* geot_ext[3];   // MIG4 metrics: Thomas factors of the extended lines per direction (or null)
  double* geot_cell[3];  // ... and of the cell-metric lines
  double* geow;          // ... work array of the line solves (extended-box layout)
  float* ig4f[3];  // mixed path: their FP32 copies (no conversions in the FP32 line solves)
  CUtensorMap ig4_tm[3][2];  // MIG4 y/z lines: TMA maps of the primitives and the temperature
  bool ig4_tma[3];           // the TMA form is used for this direction
  int* err;
  bool visc, mov, have_sponge, have_motion, metrics_ready;
  double qamb[5];
  double pref = 0.0;  // mixed path: pressure offset of the FP32 primitives (a pressure of the initial state)
  Motion motion;
  double last_fixed_dt;
  std::string last_error;
  // profiling: kernel launches issued, CUDA events around each face-flux launch
  long long launches;
  bool prof;
  std::vector<cudaEvent_t> ev;
  // pipelined host transfers (gbr_set_state_async / gbr_get_state_async): one copy stream per
  // direction and the events that order them against the context's stream (created on first use)
  cudaStream_t cs_in = nullptr, cs_out = nullptr;
  cudaEvent_t ev_in_ready = nullptr, ev_in_free = nullptr, ev_snap = nullptr, ev_out_free = nullptr;
  size_t ev_used;
};

namespace {

gbr_status fail(gbr_ctx* c, gbr_status s, const std::string& m) {
  if (c) c->last_error = m;
  g_global_error = m;
  return s;
}

gbr_status cuda_check(gbr_ctx* c, cudaError_t e, const char* what) {
  if (e != cudaSuccess) return fail(c, GBR_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return GBR_OK;
}

#define CK(expr, what)                                       \
  do {                                                       \
    gbr_status _s = cuda_check(c, (expr), what);             \
    if (_s != GBR_OK) return _s;                             \
  } while (0)
#define CKL(what)                  \
  do {                             \
    ++c->launches;                 \
    CK(cudaGetLastError(), what);  \
  } while (0)

GeoArgs geo_args(gbr_ctx* c) {
  GeoArgs G;
  G.L = c->L;
  G.nodes = c->nodes;
  G.nvel = c->nvel;
  G.xc = c->xc;
  G.vc = c->vc;
  G.xd = c->xd;
  G.mh = c->mh;
  G.det = c->det;
  G.mu = c->mu;
  G.mt = c->mt;
  for (int d = 0; d < 3; ++d) { G.fh[d] = c->fh[d]; G.fu[d] = c->fu[d]; G.ft[d] = c->ft[d]; }
  G.gcl = c->gcl;
  G.jac = c->jac;
  G.viscous = c->visc;
  G.moving = c->mov;
  return G;
}

// Unwrap periodic axes (node n = node 0 + period vector) and copy the supplied
// ghost layers of non-periodic axes into the extended node box [-E, n+E].
gbr_status build_extended(gbr_ctx* c, const double* src, bool shift, std::vector<double>& out) {
  const Layout& L = c->L;
  const int nd = L.nd;
  const int G = c->p.ghost_nodes;
  int Nn[3], off[3];
  for (int d = 0; d < 3; ++d) {
    if (d >= nd) { Nn[d] = 1; off[d] = 0; continue; }
    Nn[d] = c->p.periodic[d] ? L.n[d] + 1 : L.n[d] + 1 + 2 * G;
    off[d] = c->p.periodic[d] ? 0 : G;
  }
  const size_t NN = (size_t)Nn[0] * Nn[1] * Nn[2];
  auto sid = [&](int a, int s0, int s1, int s2) { return (size_t)a * NN + ((size_t)s2 * Nn[1] + s1) * Nn[0] + s0; };
  double per[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  if (shift) {
    double scale = 0.0;
    for (size_t m = 0; m < (size_t)nd * NN; ++m) scale = std::fmax(scale, std::fabs(src[m]));
    for (int d = 0; d < nd; ++d) {
      if (!c->p.periodic[d]) continue;
      int s0[3] = {off[0], off[1], off[2]}, s1[3] = {off[0], off[1], off[2]};
      s1[d] = L.n[d];
      for (int a = 0; a < nd; ++a) per[d][a] = src[sid(a, s1[0], s1[1], s1[2])] - src[sid(a, s0[0], s0[1], s0[2])];
      for (int s2 = 0; s2 < Nn[2]; ++s2)
        for (int s1i = 0; s1i < Nn[1]; ++s1i)
          for (int s0i = 0; s0i < Nn[0]; ++s0i) {
            int s[3] = {s0i, s1i, s2};
            if (s[d] != 0) continue;
            int t[3] = {s0i, s1i, s2};
            t[d] = L.n[d];
            for (int a = 0; a < nd; ++a) {
              double diff = src[sid(a, t[0], t[1], t[2])] - src[sid(a, s[0], s[1], s[2])];
              if (std::fabs(diff - per[d][a]) > 1e-12 * (scale + 1.0))
                return fail(c, GBR_EINVAL, "periodic axis is not closed by a constant period vector");
            }
          }
    }
  }
  out.assign((size_t)nd * L.ncount, 0.0);
  for (int mk = -L.he[2]; mk < L.nn[2] - L.he[2]; ++mk)
    for (int mj = -L.he[1]; mj < L.nn[1] - L.he[1]; ++mj)
      for (int mi = -L.he[0]; mi < L.nn[0] - L.he[0]; ++mi) {
        int m[3] = {mi, mj, mk}, s[3];
        int wraps[3] = {0, 0, 0};
        for (int d = 0; d < 3; ++d) {
          if (d >= nd) { s[d] = 0; continue; }
          if (c->p.periodic[d]) {
            int n = L.n[d];
            int base = ((m[d] % n) + n) % n;
            wraps[d] = (m[d] - base) / n;
            s[d] = base;
          } else {
            s[d] = m[d] + off[d];
          }
        }
        const long long id = nidx(L, mi, mj, mk);
        for (int a = 0; a < nd; ++a) {
          double v = src[sid(a, s[0], s[1], s[2])];
          if (shift)
            for (int d = 0; d < nd; ++d) v += wraps[d] * per[d][a];
          out[(size_t)a * L.ncount + id] = v;
        }
      }
  return GBR_OK;
}

gbr_status upload_nodes(gbr_ctx* c, const double* nodes, const double* vel) {
  std::vector<double> ext, extv;
  gbr_status s = build_extended(c, nodes, true, ext);
  if (s != GBR_OK) return s;
  CK(cudaMemcpyAsync(c->nodes, ext.data(), ext.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream), "upload nodes");
  if (c->mov) {
    if (vel) {
      s = build_extended(c, vel, false, extv);
      if (s != GBR_OK) return s;
    } else {
      extv.assign(ext.size(), 0.0);
    }
    CK(cudaMemcpyAsync(c->nvel, extv.data(), extv.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream),
       "upload node velocities");
  }
  CK(cudaStreamSynchronize(c->stream), "upload sync");  // host vectors go out of scope
  return GBR_OK;
}

// Index boxes of every launch (shared by all launch sites).
struct GeoBoxes {
  Box ext;      // centroids: cells [-E, n+E)
  Box coordd[3];  // D_d of the coordinates: [-5, n+5) along d, [-E, n+E) elsewhere
  Box metrics;  // cells [-5, n+5)
  Box faces[3]; // interfaces i+1/2, i in [-1, n-1] along d, interior elsewhere
  Box inner;    // interior cells
  Box nodes;    // extended nodes [-E, n+E]
};

GeoBoxes geo_boxes(const Layout& L) {
  GeoBoxes B;
  int elo[3], ehi[3], mlo[3], mhi[3];
  for (int e = 0; e < 3; ++e) {
    elo[e] = -L.he[e];
    ehi[e] = L.n[e] + L.he[e];
    mlo[e] = -L.cg[e];
    mhi[e] = L.n[e] + L.cg[e];
  }
  B.ext = make_box(L, elo, ehi);
  for (int d = 0; d < 3; ++d) {
    int lo[3], hi[3];
    for (int e = 0; e < 3; ++e) { lo[e] = elo[e]; hi[e] = ehi[e]; }
    lo[d] = -L.he[d] + 5;
    hi[d] = L.n[d] + L.he[d] - 5;
    B.coordd[d] = make_box(L, lo, hi);
    int flo[3] = {0, 0, 0}, fhi[3] = {L.n[0], L.n[1], L.n[2]};
    flo[d] = -1;
    fhi[d] = L.n[d];
    B.faces[d] = make_box(L, flo, fhi);
  }
  B.metrics = make_box(L, mlo, mhi);
  B.inner = pad_box(L, 0, 0);
  int lo[3], hi[3];
  for (int d = 0; d < 3; ++d) { lo[d] = -L.he[d]; hi[d] = L.n[d] + L.he[d] + 1; }
  B.nodes = make_box(L, lo, hi);
  // closed (wall-bounded) axes: geometry exists on the cells only (App. C)
  for (int a = 0; a < L.nd; ++a) {
    if (!L.closed[a]) continue;
    Box* cellb[] = {&B.ext, &B.coordd[0], &B.coordd[1], &B.coordd[2], &B.metrics};
    for (Box* b : cellb) {
      b->lo[a] = 0;
      b->hi[a] = L.n[a];
    }
    B.nodes.lo[a] = 0;
    B.nodes.hi[a] = L.n[a] + 1;
  }
  return B;
}

struct RhsBoxes {
  Box inner;
  Box halo[3];   // cross-section of axis d: padded on axes < d, interior on axes > d
  Box grad1[3];  // [-3, n+3) along e, [-1, n+1) elsewhere
  Box grad2[3];  // [-2, n+2) along e, interior elsewhere
  Box faces[3];
};

RhsBoxes rhs_boxes(const Layout& L) {
  RhsBoxes B;
  B.inner = pad_box(L, 0, 0);
  for (int d = 0; d < 3; ++d) {
    int lo[3], hi[3];
    for (int e = 0; e < 3; ++e) {
      lo[e] = (e < d) ? -H : 0;
      hi[e] = (e < d) ? L.n[e] + H : L.n[e];
    }
    lo[d] = 0;
    hi[d] = 1;
    B.halo[d] = make_box(L, lo, hi);
    int lo1[3], hi1[3], lo2[3], hi2[3];
    for (int a = 0; a < 3; ++a) {
      lo1[a] = -1; hi1[a] = L.n[a] + 1;
      lo2[a] = 0; hi2[a] = L.n[a];
    }
    lo1[d] = -3; hi1[d] = L.n[d] + 3;
    lo2[d] = -2; hi2[d] = L.n[d] + 2;
    B.grad1[d] = make_box(L, lo1, hi1);
    B.grad2[d] = make_box(L, lo2, hi2);
    int flo[3] = {0, 0, 0}, fhi[3] = {L.n[0], L.n[1], L.n[2]};
    flo[d] = -1;
    fhi[d] = L.n[d];
    B.faces[d] = make_box(L, flo, fhi);
  }
  return B;
}

// k_grad1v's launch shape for a layout: false where its rows or arrays are not 16-byte aligned
// (k_grad1t is used then).  The union U of the three first-derivative boxes, tiles of 32 x 16
// columns, chunks of zchunk planes: zchunk = 0 picks them so that the launch has about
// GBR_G1V_BLOCKS blocks per SM, zchunk < 0 balances chunks of at most -zchunk planes.
struct G1VPlan {
  Box U;
  int tiles_x, tiles_y, zchunk, chunks, nf;
  long long blocks() const { return (long long)tiles_x * tiles_y * chunks * nf; }
};
bool g1v_plan(const Layout& L, const RhsBoxes& B, const void* prim, const void* temp, const void* const g1[3], bool visc,
              int zchunk, G1VPlan& P) {
  auto al16 = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; };
  if (L.nd != 3 || L.ps[1] % 4 != 0 || !al16(prim) || (visc && !al16(temp)) || !al16(g1[0]) || !al16(g1[1]) ||
      !al16(g1[2]))
    return false;
  for (int d = 0; d < 3; ++d) {
    P.U.lo[d] = std::min(B.grad1[0].lo[d], std::min(B.grad1[1].lo[d], B.grad1[2].lo[d]));
    P.U.hi[d] = std::max(B.grad1[0].hi[d], std::max(B.grad1[1].hi[d], B.grad1[2].hi[d]));
  }
  P.nf = L.nv + (visc ? 1 : 0);
  P.tiles_x = (P.U.hi[0] + L.hp[0] + 4 * kGVX - 1) / (4 * kGVX);
  P.tiles_y = (P.U.hi[1] - P.U.lo[1] + kGVY - 1) / kGVY;
  const int nzu = P.U.hi[2] - P.U.lo[2];
  if (zchunk < 0) {
    const int chunks = (nzu - zchunk - 1) / -zchunk;
    zchunk = (nzu + chunks - 1) / chunks;
  } else if (zchunk == 0) {
    const int pairs = P.tiles_x * P.tiles_y * P.nf;
    const int chunks = std::max(1, std::min(nzu, (GBR_G1V_BLOCKS * device_sms() + pairs - 1) / pairs));
    zchunk = (nzu + chunks - 1) / chunks;
  }
  P.zchunk = zchunk;
  P.chunks = (nzu + zchunk - 1) / zchunk;
  return true;
}

DtArgs dt_args(gbr_ctx* c);

// the box b with its extent along d reduced to the single index 0 (one thread per line along d)
Box cross_section(Box b, int d) {
  b.lo[d] = 0;
  b.hi[d] = 1;
  return b;
}

// MIG4 metrics (Sec. 7 steps 2-3 with IG4 line solves; App. C on wall-bounded axes)
gbr_status run_geometry_ig4(gbr_ctx* c, const GeoArgs& G, const GeoBoxes& B, cudaStream_t st) {
  const Layout& L = c->L;
  constexpr int kLineBlock = 64;
  for (int d = 0; d < L.nd; ++d) {
    if (L.closed[d]) {
      k_coordd1<<<grid_of(B.coordd[d], kBlock), kBlock, 0, st>>>(G, d, B.coordd[d]);
      CKL("k_coordd1");
    } else {
      const Box xs = cross_section(B.ext, d);
      k_ig4_coordd<<<grid_of(xs, kLineBlock), kLineBlock, 0, st>>>(G, d, xs, c->geot_ext[d], c->geow);
      CKL("k_ig4_coordd");
    }
  }
  if (L.nd == 3)
    for (int phase = 0; phase < 2; ++phase)
      for (int s = 0; s < 3; ++s) {
        const Box xs = cross_section(B.metrics, s);
        k_ig4_metric_terms<<<grid_of(xs, kLineBlock), kLineBlock, 0, st>>>(G, s, phase, xs, c->geot_ext[s], c->geow);
        CKL("k_ig4_metric_terms");
      }
  k_metrics_given<<<grid_of(B.metrics, kBlock), kBlock, 0, st>>>(G, B.metrics);
  CKL("k_metrics_given");
  for (int d = 0; d < L.nd; ++d) {
    const Box xs = cross_section(B.inner, d);
    k_ig4_face_metrics<<<grid_of(xs, kLineBlock), kLineBlock, 0, st>>>(G, d, xs, c->geot_cell[d], c->geow);
    CKL("k_ig4_face_metrics");
  }
  return GBR_OK;
}

// FP64 path on a static mesh: the time step's metric norms (after J, k_gcl)
__global__ void k_dt_geo(DtArgs D, double* gdt, Box b) {
  BOX_THREAD(b);
  body_dt_geo(D, gdt, i, j, k);
}

// FP64 path: the interface geometry of every direction, after the interface metrics
gbr_status launch_face_geo(gbr_ctx* c, const GeoArgs& G, const GeoBoxes& B, cudaStream_t st) {
  if (!c->fg[0]) return GBR_OK;
  FaceGeoOut O;
  unsigned gmax = 0;
  for (int d = 0; d < 3; ++d) {
    O.fg[d] = c->fg[d];
    if (d < c->L.nd) gmax = std::max(gmax, grid_of(B.faces[d], kBlock));
  }
  k_face_geo<<<dim3(gmax, c->L.nd), kBlock, 0, st>>>(G, O, B.faces[0], B.faces[1], B.faces[2]);
  CKL("k_face_geo");
  return GBR_OK;
}

gbr_status run_geometry(gbr_ctx* c, cudaStream_t st) {
  const Layout& L = c->L;
  GeoArgs G = geo_args(c);
  const GeoBoxes B = geo_boxes(L);
  k_centroid<<<grid_of(B.ext, kBlock), kBlock, 0, st>>>(G, B.ext);
  CKL("k_centroid");
  if (c->p.gradient_scheme == GBR_GRAD_MIG4) {
    gbr_status s4 = run_geometry_ig4(c, G, B, st);
    if (s4 != GBR_OK) return s4;
  } else {
    unsigned gmax = 0;
    for (int d = 0; d < L.nd; ++d) gmax = std::max(gmax, grid_of(B.coordd[d], kBlock));
    k_coordd<<<dim3(gmax, L.nd), kBlock, 0, st>>>(G, B.coordd[0], B.coordd[1], B.coordd[2]);
    CKL("k_coordd");
    k_metrics<<<grid_of(B.metrics, kBlock), kBlock, 0, st>>>(G, B.metrics);
    CKL("k_metrics");
    gmax = 0;
    for (int d = 0; d < L.nd; ++d) gmax = std::max(gmax, grid_of(B.faces[d], kBlock));
    k_face_metrics<<<dim3(gmax, L.nd), kBlock, 0, st>>>(G, B.faces[0], B.faces[1], B.faces[2]);
    CKL("k_face_metrics");
  }
  {
    gbr_status sg = launch_face_geo(c, G, B, st);
    if (sg != GBR_OK) return sg;
  }
  k_gcl<<<grid_of(B.inner, kBlock), kBlock, 0, st>>>(G, B.inner);
  CKL("k_gcl");
  if (c->gdt) {
    k_dt_geo<<<grid_of(B.inner, kBlock), kBlock, 0, st>>>(dt_args(c), c->gdt, B.inner);
    CKL("k_dt_geo");
  }
  if (c->p.precision == GBR_PREC_MIXED) {
    // FP32 copies of the interface metrics (whole slots: all directions at once)
    const Plan& P = c->plan;
    const int slots[3][2] = {{SL_FH, SL_FH32}, {SL_FU, SL_FU32}, {SL_FT, SL_FT32}};
    for (auto& sl : slots) {
      const long long n = (long long)(P.len[sl[1]] / sizeof(float));
      if (n == 0) continue;
      k_to_f32<<<(unsigned)((n + kBlock - 1) / kBlock), kBlock, 0, st>>>(
          (const double*)(c->ws + P.off[sl[0]]), (float*)(c->ws + P.off[sl[1]]), n);
      CKL("k_to_f32");
    }
    // and of the cell metrics and J the time step reads
    k_dt_f32<<<grid_of(B.inner, kBlock), kBlock, 0, st>>>(dt_args(c), c->mh32, c->mt32, c->jac32, B.inner);
    CKL("k_dt_f32");
  }
  return GBR_OK;
}

gbr_status run_geometry(gbr_ctx* c) { return run_geometry(c, c->stream); }

gbr_status run_motion(gbr_ctx* c, double stage_c, cudaStream_t st) {
  const Box bn = geo_boxes(c->L).nodes;
  k_motion<<<grid_of(bn, kBlock), kBlock, 0, st>>>(c->L, c->motion, c->scal, stage_c, c->nodes, c->nvel, bn);
  CKL("k_motion");
  return GBR_OK;
}
gbr_status run_motion(gbr_ctx* c, double stage_c) { return run_motion(c, stage_c, c->stream); }

template <class R>
RhsArgsT<R> rhs_args_r(gbr_ctx* c, const double* q) {
  RhsArgsT<R> A;
  A.L = c->L;
  A.ph = c->ph;
  // the first derivatives carry kE6Scale with E6 (stencil_E6x60), 1 with IG4 (the line solves)
  A.pr = phys_r<R>(c->ph, c->p.gradient_scheme == GBR_GRAD_MIG4 ? 1.0 : kE6Scale);
  A.q = q;
  A.prim = static_cast<R*>(c->prim);
  A.temp = static_cast<R*>(c->temp);
  for (int d = 0; d < 3; ++d) {
    A.g1[d] = static_cast<R*>(c->g1[d]);
    A.g2[d] = static_cast<R*>(c->g2[d]);
    if constexpr (sizeof(R) == 4) {
      A.fh[d] = c->fh32[d];
      A.fu[d] = c->fu32[d];
      A.ft[d] = c->ft32[d];
    } else {
      A.fh[d] = c->fh[d];
      A.fu[d] = c->fu[d];
      A.ft[d] = c->ft[d];
    }
    A.flux[d] = static_cast<R*>(c->flux[d]);
    if constexpr (sizeof(R) == sizeof(double)) A.fg[d] = c->fg[d];
    else A.fg[d] = nullptr;
  }
  A.inflow = c->inflow;
  for (int d = 0; d < 3; ++d)
    for (int s = 0; s < 2; ++s) A.bc[d][s] = c->p.bc[d][s];
  A.viscous = c->visc;
  A.pref = (sizeof(R) == 4) ? c->pref : 0.0;
  A.pref_r = R(A.pref);
  return A;
}
RhsArgs rhs_args(gbr_ctx* c, const double* q) { return rhs_args_r<double>(c, q); }

gbr_status prof_event(gbr_ctx* c) {
  if (c->ev_used == c->ev.size()) {
    cudaEvent_t e;
    CK(cudaEventCreate(&e), "event create");
    c->ev.push_back(e);
  }
  CK(cudaEventRecord(c->ev[c->ev_used++], c->stream), "event record");
  return GBR_OK;
}

template <int ND, class R>
gbr_status launch_face(gbr_ctx* c, const RhsArgsT<R>& A, int d, const Box& b) {
  cudaStream_t st = c->stream;
  if (c->prof) {
    gbr_status s0 = prof_event(c);
    if (s0 != GBR_OK) return s0;
  }
  // one instantiation per sweep direction (d fixed at compile time)
  auto launch = [&](auto dd) {
    constexpr int D = decltype(dd)::value, BS = face_bs<D>();
    const unsigned g = face_grid<R, ND, D>(b);
    if (c->visc) {
      if (c->mov) k_face<ND, true, true, R, D><<<g, BS, 0, st>>>(A, d, b);
      else k_face<ND, true, false, R, D><<<g, BS, 0, st>>>(A, d, b);
    } else {
      if (c->mov) k_face<ND, false, true, R, D><<<g, BS, 0, st>>>(A, d, b);
      else k_face<ND, false, false, R, D><<<g, BS, 0, st>>>(A, d, b);
    }
  };
  if (d == 0) launch(std::integral_constant<int, 0>{});
  else if (d == 1) launch(std::integral_constant<int, 1>{});
  else if constexpr (ND == 3) launch(std::integral_constant<int, 2>{});
  CKL("k_face");
  if (c->prof) return prof_event(c);
  return GBR_OK;
}

// the shared-memory opt-in of the MIG4 line-solve kernels (above the 48 KB default), once per
// instantiation; also called at gbr_create, so that no first launch sets it inside a graph capture
template <int ND, class R>
void ig4_attributes() {
  static bool done = false;
  if (done) return;
  cudaFuncSetAttribute(k_ig4t<ND, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kIg4SmemMax);
  cudaFuncSetAttribute(k_ig4s<ND, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kIg4SmemMax);
  done = true;
}

// MIG4 first derivatives of every direction (Eq. IG4_grads): one line solve per grid line, on a
// tile staged by TMA (y/z lines), by cp.async (x-lines and the fallback) or in global memory
template <int ND, class R>
gbr_status launch_ig4_grads(gbr_ctx* c, const RhsArgsT<R>& A, cudaStream_t st) {
  ig4_attributes<ND, R>();
  const Layout& L = c->L;
  const RhsBoxes B = rhs_boxes(L);
  const int nf = L.nv + (c->visc ? 1 : 0);
  for (int e = 0; e < ND; ++e) {
    Box lines = B.grad1[e];
    lines.lo[e] = 0;
    lines.hi[e] = 1;
    const R* table;
    if constexpr (sizeof(R) == sizeof(float)) table = c->ig4f[e];
    else table = c->ig4[e];
    const bool per = L.per[e] != 0;
    const int tlen = (int)ig4_table_len(L.n[e], per);
    const size_t smem = ig4_smem_bytes<R>(L.n[e], per);
    if (c->ig4_tma[e]) {
      const int bx = (e == 1) ? 2 : 1;
      const int x0p = (lines.lo[0] + L.hp[0]) & ~3;
      const int tiles = (lines.hi[0] + L.hp[0] - x0p + kIg4Lines - 1) / kIg4Lines;
      const int nb = lines.hi[bx] - lines.lo[bx];
      k_ig4t<ND, R><<<dim3((unsigned)(tiles * nb), nf), kIg4Lines, ig4t_smem_bytes<R>(L.n[e], per), st>>>(
          A, e, lines, table, tlen, x0p, c->ig4_tm[e][0], c->ig4_tm[e][1], c->err);
    } else if (smem <= kIg4SmemMax) {
      const int a = (e == 0) ? 1 : 0, bx = 3 - e - a;
      const int na = lines.hi[a] - lines.lo[a], nb = lines.hi[bx] - lines.lo[bx];
      const unsigned tiles = (unsigned)((na + kIg4Lines - 1) / kIg4Lines) * (unsigned)nb;
      k_ig4s<ND, R><<<dim3(tiles, nf), kIg4Lines, smem, st>>>(A, e, lines, table, ig4_srow(L.n[e]), tlen);
    } else {
      k_ig4<ND, R><<<dim3(grid_of(lines, 128), nf), 128, 0, st>>>(A, e, lines, table);
    }
    CKL("k_ig4");
  }
  return GBR_OK;
}

// one evaluation of L(qs [+ dq_in]): out = L (mode 0) or the RK combination (mode 1), the latter
// in increments when dq_in / dq_out are given (mixed path, body_update)
template <int ND, class R>
gbr_status run_rhs_nd(gbr_ctx* c, const double* qs, const double* q0, double* out, int mode, double ca, double cb,
                      double cc, const float* dq_in, float* dq_out) {
  const Layout& L = c->L;
  cudaStream_t st = c->stream;
  const RhsArgsT<R> A = rhs_args_r<R>(c, qs);
  const RhsBoxes B = rhs_boxes(L);
  const Box bi = B.inner;
  // primitives and all ghost layers in one pass over the padded box
  const Box pad = pad_box(L, H, H);
  bool special = false;  // an inflow or wall boundary on some non-periodic axis
  for (int d = 0; d < ND; ++d)
    if (!L.per[d])
      special |= A.bc[d][0] == 2 || A.bc[d][0] == 3 || A.bc[d][1] == 3;
  if (special) k_prim_halo<ND, R, true><<<grid_of(pad, kBlock), kBlock, 0, st>>>(A, qs, dq_in, pad);
  else k_prim_halo<ND, R, false><<<grid_of(pad, kBlock), kBlock, 0, st>>>(A, qs, dq_in, pad);
  CKL("k_prim_halo");
  unsigned g1 = 0, g2 = 0;
  for (int e = 0; e < ND; ++e) {
    g1 = std::max(g1, grid_of(B.grad1[e], kBlock));
    g2 = std::max(g2, grid_of(B.grad2[e], kBlock));
  }
  if (c->p.gradient_scheme == GBR_GRAD_MIG4) {
    gbr_status sg = launch_ig4_grads<ND, R>(c, A, st);
    if (sg != GBR_OK) return sg;
  } else {
    if constexpr (ND == 3 && sizeof(R) == sizeof(float)) {
      // one z-marching block per 32 x 8 tile of the union of the three boxes and chunk of planes
      // (FP32; the FP64 pass is bound by the FP64 pipe, where the per-cell kernel measured faster)
      Box U;
      for (int d = 0; d < 3; ++d) {
        U.lo[d] = std::min(B.grad1[0].lo[d], std::min(B.grad1[1].lo[d], B.grad1[2].lo[d]));
        U.hi[d] = std::max(B.grad1[0].hi[d], std::max(B.grad1[1].hi[d], B.grad1[2].hi[d]));
      }
      const int nf = L.nv + (c->visc ? 1 : 0);
      const int tiles_x = (U.hi[0] - U.lo[0] + kG1TX - 1) / kG1TX, tiles_y = (U.hi[1] - U.lo[1] + kG1TY - 1) / kG1TY;
      const int nzu = U.hi[2] - U.lo[2];
      // four cells per thread where the padded rows and the arrays sit on 16-byte boundaries
      const void* g1p[3] = {A.g1[0], A.g1[1], A.g1[2]};
      G1VPlan P;
      if (g1v_plan(L, B, A.prim, A.temp, g1p, c->visc, 0, P)) {
        k_grad1v<<<dim3((unsigned)(P.tiles_x * P.tiles_y * P.chunks), P.nf), kGVX * kGVY, 0, st>>>(
            A, P.U, B.grad1[0], B.grad1[1], B.grad1[2], P.tiles_x, P.tiles_y, P.zchunk);
      } else {
        // chunks of planes: about kG1Waves waves of resident blocks (8 per SM)
        const int fb = (nf + kG1Fields - 1) / kG1Fields;  // field groups
        const int pairs = tiles_x * tiles_y * fb;
        const int chunks = std::max(1, std::min(nzu, (kG1Waves * device_sms() * 8 + pairs - 1) / pairs));
        const int zchunk = (nzu + chunks - 1) / chunks;
        const unsigned blocks = (unsigned)(tiles_x * tiles_y * ((nzu + zchunk - 1) / zchunk));
        k_grad1t<R, kG1Fields><<<dim3(blocks, fb), kG1TX * kG1TY, 0, st>>>(A, U, B.grad1[0], B.grad1[1], B.grad1[2],
                                                                           tiles_x, tiles_y, zchunk, nf);
      }
    } else {
      k_grad1<ND, R><<<g1 * ND, kBlock, 0, st>>>(A, B.grad1[0], B.grad1[1], B.grad1[2]);
    }
    CKL("k_grad1");
  }
  if constexpr (!kFaceFormsG2<R>) {
    k_grad2<ND, R><<<g2 * ND, kBlock, 0, st>>>(A, B.grad2[0], B.grad2[1], B.grad2[2]);
    CKL("k_grad2");
  }
  for (int d = 0; d < ND; ++d) {
    gbr_status s = launch_face<ND, R>(c, A, d, B.faces[d]);
    if (s != GBR_OK) return s;
  }
  UpdArgsT<R> U;
  U.L = L;
  for (int d = 0; d < 3; ++d) U.flux[d] = static_cast<const R*>(c->flux[d]);
  U.qs = qs;
  U.q0 = q0;
  U.out = out;
  U.jac = c->jac;
  U.jac32 = c->jac32;
  U.gcl = c->gcl;
  U.sigma = c->have_sponge ? c->sigma : nullptr;
  for (int v = 0; v < 5; ++v) U.qamb[v] = c->qamb[v];
  U.dt = c->scal + S_DT;
  U.ca = ca;
  U.cb = cb;
  U.cc = cc;
  U.mode = mode;
  U.dq_in = dq_in;
  U.dq_out = dq_out;
  if (c->mov) k_update<ND, true, R><<<grid_of(bi, kBlock), kBlock, 0, st>>>(U, bi, c->err);
  else if (U.sigma) k_update<ND, false, R, true><<<grid_of(bi, kBlock), kBlock, 0, st>>>(U, bi, c->err);
  else k_update<ND, false, R, false><<<grid_of(bi, kBlock), kBlock, 0, st>>>(U, bi, c->err);
  CKL("k_update");
  return GBR_OK;
}

gbr_status run_rhs(gbr_ctx* c, const double* qs, const double* q0, double* out, int mode, double ca, double cb,
                   double cc, const float* dq_in = nullptr, float* dq_out = nullptr) {
  if (c->p.precision == GBR_PREC_MIXED)
    return c->L.nd == 3 ? run_rhs_nd<3, float>(c, qs, q0, out, mode, ca, cb, cc, dq_in, dq_out)
                        : run_rhs_nd<2, float>(c, qs, q0, out, mode, ca, cb, cc, dq_in, dq_out);
  return c->L.nd == 3 ? run_rhs_nd<3, double>(c, qs, q0, out, mode, ca, cb, cc, nullptr, nullptr)
                      : run_rhs_nd<2, double>(c, qs, q0, out, mode, ca, cb, cc, nullptr, nullptr);
}

// the SSP-RK3 stages as Q^n plus FP32 increments: mixed path on a static mesh (no GCL term, no
// motion or geometry change within the step)
bool rk_in_increments(const gbr_ctx* c) {
  return c->p.precision == GBR_PREC_MIXED && !c->mov && !c->have_motion && c->jac32;
}

DtArgs dt_args(gbr_ctx* c) {
  DtArgs D;
  D.L = c->L;
  D.ph = c->ph;
  D.q = c->q[0];
  D.mh = c->mh;
  D.mt = c->mov ? c->mt : nullptr;
  D.jac = c->jac;
  D.mh32 = c->mh32;
  D.mt32 = c->mov ? c->mt32 : nullptr;
  D.jac32 = c->jac32;
  D.gdt = c->gdt;
  return D;
}

gbr_status run_dt(gbr_ctx* c, double cfl) {
  const Layout& L = c->L;
  const DtArgs D = dt_args(c);
  Box bi = pad_box(L, 0, 0);
  unsigned long long* bits = reinterpret_cast<unsigned long long*>(c->scal + S_DTMIN);
  k_dt_init<<<1, 1, 0, c->stream>>>(bits);
  CKL("k_dt_init");
  const unsigned g = grid_of(bi, kBlock);
  cudaStream_t st = c->stream;
  if (c->p.precision == GBR_PREC_MIXED) {
    if (L.nd == 3) k_dt<3, float><<<g, kBlock, 0, st>>>(D, bi, bits);
    else k_dt<2, float><<<g, kBlock, 0, st>>>(D, bi, bits);
  } else {
    if (D.gdt) {
      if (L.nd == 3) k_dt<3, double, true><<<g, kBlock, 0, st>>>(D, bi, bits);
      else k_dt<2, double, true><<<g, kBlock, 0, st>>>(D, bi, bits);
    } else {
      if (L.nd == 3) k_dt<3, double><<<g, kBlock, 0, st>>>(D, bi, bits);
      else k_dt<2, double><<<g, kBlock, 0, st>>>(D, bi, bits);
    }
  }
  CKL("k_dt");
  k_dt_final<<<1, 1, 0, c->stream>>>(c->scal, bits, cfl);
  CKL("k_dt_final");
  return GBR_OK;
}

void carve(gbr_ctx* c) {
  const Plan& P = c->plan;
  const Layout& L = c->L;
  auto ptr = [&](int slot) -> double* { return P.len[slot] ? (double*)(c->ws + P.off[slot]) : nullptr; };
  for (int s = 0; s < 3; ++s) c->q[s] = ptr(SL_Q0 + s);
  // arrays of the path's type: offsets in bytes of that type
  const size_t ER = elem_r(&c->p);
  auto rptr = [&](int slot, size_t elems) -> void* { return P.len[slot] ? c->ws + P.off[slot] + ER * elems : nullptr; };
  c->prim = rptr(SL_PRIM, 0);
  c->temp = rptr(SL_TEMP, 0);
  c->gdt = ptr(SL_GDT);
  const int nv = L.nv, nd = L.nd;
  const int n1 = nv + (c->visc ? 1 : 0);
  size_t foff = 0;
  for (int d = 0; d < 3; ++d) {
    c->g1[d] = (d < nd) ? rptr(SL_G1, (size_t)d * n1 * L.pcount) : nullptr;
    c->g2[d] = (d < nd && c->p.precision != GBR_PREC_MIXED) ? rptr(SL_G2, (size_t)d * nv * L.pcount) : nullptr;
    c->flux[d] = (d < nd) ? rptr(SL_FLUX, (size_t)nv * foff) : nullptr;
    c->fh[d] = (d < nd) ? ptr(SL_FH) + (size_t)nd * foff : nullptr;
    c->fu[d] = (d < nd && c->visc) ? ptr(SL_FU) + (size_t)nd * nd * foff : nullptr;
    c->ft[d] = (d < nd && c->mov) ? ptr(SL_FT) + foff : nullptr;
    c->fg[d] = (d < nd && P.len[SL_FG]) ? ptr(SL_FG) + (size_t)fg_count(c->visc) * foff : nullptr;
    auto fptr = [&](int slot, size_t elems) -> float* {
      return P.len[slot] ? (float*)(c->ws + P.off[slot]) + elems : nullptr;
    };
    c->fh32[d] = (d < nd) ? fptr(SL_FH32, (size_t)nd * foff) : nullptr;
    c->fu32[d] = (d < nd && c->visc) ? fptr(SL_FU32, (size_t)nd * nd * foff) : nullptr;
    c->ft32[d] = (d < nd && c->mov) ? fptr(SL_FT32, foff) : nullptr;
    if (d < nd) foff += (size_t)L.fcount[d];
  }
  c->nodes = ptr(SL_NODES);
  c->nvel = ptr(SL_NVEL);
  c->xc = ptr(SL_XC);
  c->vc = ptr(SL_VC);
  c->xd = ptr(SL_XD);
  c->mh = ptr(SL_MH);
  c->det = ptr(SL_DET);
  c->mu = ptr(SL_MU);
  c->mt = ptr(SL_MT);
  c->gcl = ptr(SL_GCL);
  c->jac = ptr(SL_JAC);
  {
    auto f32p = [&](int slot) -> float* { return P.len[slot] ? (float*)(c->ws + P.off[slot]) : nullptr; };
    c->mh32 = f32p(SL_MH32);
    c->mt32 = f32p(SL_MT32);
    c->jac32 = f32p(SL_JAC32);
  }
  c->sigma = ptr(SL_SIGMA);
  c->inflow = ptr(SL_INFLOW);
  c->scal = ptr(SL_SCAL);
  c->err = (int*)(c->ws + P.off[SL_ERR]);
  {
    size_t toff = 0;
    for (int d = 0; d < 3; ++d) {
      c->ig4[d] = nullptr;
      c->ig4f[d] = nullptr;
      if (d < L.nd && P.len[SL_IG4]) {
        c->ig4[d] = (double*)(c->ws + P.off[SL_IG4]) + toff;
        if (P.len[SL_IG4F]) c->ig4f[d] = (float*)(c->ws + P.off[SL_IG4F]) + toff;
        toff += (size_t)ig4_table_len(L.n[d], L.per[d] != 0);
      }
    }
  }
  {
    size_t goff = 0;
    for (int d = 0; d < 3; ++d) {
      c->geot_ext[d] = c->geot_cell[d] = nullptr;
      if (d < L.nd && P.len[SL_GEOT]) {
        c->geot_ext[d] = (double*)(c->ws + P.off[SL_GEOT]) + goff;
        goff += 2 * (size_t)(L.n[d] + 2 * L.he[d]);
        c->geot_cell[d] = (double*)(c->ws + P.off[SL_GEOT]) + goff;
        goff += 2 * (size_t)(L.n[d] + 2 * L.cg[d]);
      }
    }
    c->geow = ptr(SL_GEOW);
  }
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link against the driver library)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<EncodeTiledFn>(f);
  }();
  return fn;
}

// TMA maps of the MIG4 y- and z-line tiles (k_ig4t): the primitives as a 4D tensor {px, py, pz, nv}
// and the temperature as a 3D one, each with the box {32 along x, the padded line along e}.  A
// direction keeps the staged plain-load kernel when a TMA rule does not hold: the row pitch and
// the base addresses must be multiples of 16 bytes, a box extent at most 256.
void ig4_encode_maps(gbr_ctx* c) {
  const Layout& L = c->L;
  const size_t es = elem_r(&c->p);
  EncodeTiledFn enc = encode_tiled();
  for (int e = 0; e < 3; ++e) c->ig4_tma[e] = false;
  const bool aligned = ((uintptr_t)c->prim % 16 == 0) && (!c->visc || (uintptr_t)c->temp % 16 == 0) &&
                       ((size_t)L.pn[0] * es) % 16 == 0;
  if (!enc || !aligned) return;
  const CUtensorMapDataType dt = (es == 4) ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
  const cuuint64_t dims[4] = {(cuuint64_t)L.pn[0], (cuuint64_t)L.pn[1], (cuuint64_t)L.pn[2], (cuuint64_t)L.nv};
  const cuuint64_t strides[3] = {(cuuint64_t)(L.ps[1] * es), (cuuint64_t)(L.ps[2] * es), (cuuint64_t)(L.pcount * es)};
  const cuuint32_t ones[4] = {1, 1, 1, 1};
  for (int e = 1; e < L.nd; ++e) {
    const int M = L.n[e] + 2 * H;
    if (M > 256) continue;
    cuuint32_t box[4] = {(cuuint32_t)kIg4Lines, 1, 1, 1};
    box[e] = (cuuint32_t)M;
    bool ok = enc(&c->ig4_tm[e][0], dt, 4, c->prim, dims, strides, box, ones, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    if (ok && c->visc)
      ok = enc(&c->ig4_tm[e][1], dt, 3, c->temp, dims, strides, box, ones, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    else if (ok)
      c->ig4_tm[e][1] = c->ig4_tm[e][0];  // never read (no temperature field without viscosity)
    c->ig4_tma[e] = ok;
  }
}

Phys phys_of(const gbr_params* p) {
  Phys ph;
  ph.gamma = p->gamma;
  ph.gm1 = p->gamma - 1.0;
  ph.igm1 = 1.0 / (p->gamma - 1.0);
  ph.viscous = p->reynolds > 0.0;
  ph.mu_ref = ph.viscous ? 1.0 / p->reynolds : 0.0;
  ph.sutherland = p->sutherland_s > 0.0;
  ph.suth_s = p->sutherland_s;
  ph.it_ref = p->t_ref > 0.0 ? 1.0 / p->t_ref : 1.0;
  ph.alpha_d = p->alpha_damping;
  ph.mp_alpha = p->mp_alpha;
  ph.mp_beta = p->mp_beta;
  ph.mp_eps = p->mp_eps;
  ph.kfac = ph.viscous ? p->gamma / ((p->gamma - 1.0) * p->prandtl) : 0.0;
  ph.dt_visc_fac = ph.viscous ? std::fmax(4.0 / 3.0, p->gamma / p->prandtl) : 0.0;
  return ph;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

size_t gbr_workspace_bytes(const gbr_params* p) {
  std::string why;
  if (!valid_params(p, why)) { g_global_error = why; return 0; }
  Layout L = layout_of(p);
  return plan_of(p, L).total;
}

gbr_status gbr_create(const gbr_params* p, const double* nodes, const double* node_vel, void* d_workspace,
                      size_t ws_bytes, void* stream, gbr_ctx** out) {
  if (!out) return fail(nullptr, GBR_EINVAL, "null output pointer");
  *out = nullptr;
  std::string why;
  if (!valid_params(p, why)) return fail(nullptr, GBR_EINVAL, why);
  if (!nodes) return fail(nullptr, GBR_EINVAL, "null node array");
  if (!d_workspace) return fail(nullptr, GBR_EINVAL, "null workspace");
  if (((uintptr_t)d_workspace & 255) != 0) return fail(nullptr, GBR_EINVAL, "workspace must be 256-byte aligned");
  Layout L = layout_of(p);
  Plan P = plan_of(p, L);
  if (ws_bytes < P.total) return fail(nullptr, GBR_ENOMEM, "workspace smaller than gbr_workspace_bytes");
  gbr_ctx* c = new gbr_ctx();
  c->p = *p;
  if (p->ndim == 2) c->p.n[2] = 1;
  c->L = L;
  c->ph = phys_of(p);
  c->stream = (cudaStream_t)stream;
  c->ws = (char*)d_workspace;
  c->ws_bytes = ws_bytes;
  c->plan = P;
  c->visc = p->reynolds > 0.0;
  c->mov = p->moving != 0;
  c->have_sponge = false;
  c->have_motion = false;
  c->metrics_ready = false;
  c->last_fixed_dt = 0.0;
  c->launches = 0;
  c->prof = false;
  c->ev_used = 0;
  for (int v = 0; v < 5; ++v) c->qamb[v] = 0.0;
  carve(c);
  cudaError_t e = cudaMemsetAsync(c->ws, 0, P.total, c->stream);
  if (e != cudaSuccess) {
    gbr_status s = fail(c, GBR_ECUDA, std::string("clear workspace: ") + cudaGetErrorString(e));
    delete c;
    return s;
  }
  if (p->gradient_scheme == GBR_GRAD_MIG4) {
    if (L.nd == 3) {
      if (p->precision == GBR_PREC_MIXED) ig4_attributes<3, float>();
      else ig4_attributes<3, double>();
    } else {
      if (p->precision == GBR_PREC_MIXED) ig4_attributes<2, float>();
      else ig4_attributes<2, double>();
    }
    ig4_encode_maps(c);
    for (int d = 0; d < L.nd; ++d) {
      if (!L.closed[d]) {  // the metric line solves (extended lines, cell-metric lines)
        k_ig4_geo_factor<<<1, 1, 0, c->stream>>>(c->geot_ext[d], L.n[d] + 2 * L.he[d]);
        k_ig4_geo_factor<<<1, 1, 0, c->stream>>>(c->geot_cell[d], L.n[d] + 2 * L.cg[d]);
      }
      k_ig4_factor<<<1, 1, 0, c->stream>>>(c->ig4[d], L.n[d], L.per[d]);
      if (c->ig4f[d]) {
        const long long n = ig4_table_len(L.n[d], L.per[d] != 0);
        k_to_f32<<<(unsigned)((n + kBlock - 1) / kBlock), kBlock, 0, c->stream>>>(c->ig4[d], c->ig4f[d], n);
      }
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) {
      gbr_status s = fail(c, GBR_ECUDA, std::string("MIG4 factors: ") + cudaGetErrorString(e));
      delete c;
      return s;
    }
  }
  gbr_status s = upload_nodes(c, nodes, node_vel);
  if (s != GBR_OK) {
    g_global_error = c->last_error;
    delete c;
    return s;
  }
  *out = c;
  return GBR_OK;
}

gbr_status gbr_compute_metrics(gbr_ctx* c) {
  if (!c) return fail(nullptr, GBR_EINVAL, "null context");
  gbr_status s = run_geometry(c);
  if (s != GBR_OK) return s;
  c->metrics_ready = true;
  return GBR_OK;
}

gbr_status gbr_move_mesh(gbr_ctx* c, const double* nodes, const double* node_vel) {
  if (!c || !nodes) return fail(c, GBR_EINVAL, "null argument");
  if (node_vel && !c->mov) return fail(c, GBR_EINVAL, "node velocities need params.moving = 1");
  c->have_motion = false;
  gbr_status s = upload_nodes(c, nodes, node_vel);
  if (s != GBR_OK) return s;
  return gbr_compute_metrics(c);
}

gbr_status gbr_set_motion(gbr_ctx* c, const gbr_motion* m, double t0) {
  if (!c || !m) return fail(c, GBR_EINVAL, "null argument");
  if (!c->mov) return fail(c, GBR_EINVAL, "a motion needs params.moving = 1");
  for (int d = 0; d < c->L.nd; ++d)
    if (!c->p.periodic[d]) return fail(c, GBR_EINVAL, "analytic motion needs periodic axes");
  Motion M;
  for (int a = 0; a < 3; ++a) {
    M.origin[a] = m->origin[a];
    M.h[a] = m->h[a];
    M.amp[a] = m->amp[a];
    for (int b = 0; b < 3; ++b) M.k[a][b] = m->k[a][b];
  }
  M.omega = m->omega;
  c->motion = M;
  c->have_motion = true;
  k_set_scalar<<<1, 1, 0, c->stream>>>(c->scal, S_T, t0);
  CKL("k_set_scalar");
  gbr_status s = run_motion(c, 0.0);
  if (s != GBR_OK) return s;
  return gbr_compute_metrics(c);
}

gbr_status gbr_set_state(gbr_ctx* c, const double* q, int on_device) {
  if (!c || !q) return fail(c, GBR_EINVAL, "null argument");
  const size_t bytes = sizeof(double) * c->L.nv * c->L.ncells;
  CK(cudaMemcpyAsync(c->q[0], q, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream),
     "set state");
  if (!on_device) CK(cudaStreamSynchronize(c->stream), "set state sync");
  if (c->p.precision == GBR_PREC_MIXED) {
    // the FP32 primitives store p - pref with pref the pressure of the first cell (any constant is
    // exact; one of the flow's own pressures keeps the stored differences' digits)
    const int nv = c->L.nv;
    double q0[5];
    for (int v = 0; v < nv; ++v)
      CK(cudaMemcpyAsync(q0 + v, c->q[0] + (size_t)v * c->L.ncells, sizeof(double), cudaMemcpyDeviceToHost,
                         c->stream),
         "read first cell");
    CK(cudaStreamSynchronize(c->stream), "read first cell sync");
    double ke = 0.0;
    for (int a = 0; a < c->L.nd; ++a) ke += q0[1 + a] * q0[1 + a] / q0[0];
    const double p0 = (c->p.gamma - 1.0) * (q0[nv - 1] - 0.5 * ke);
    // rounded to FP32, so that the FP64 primitive pass and the FP32 kernels use the same number
    c->pref = std::isfinite(p0) && std::fabs(p0) < 1e38 ? (double)(float)p0 : 0.0;
  }
  return GBR_OK;
}

gbr_status gbr_get_state(gbr_ctx* c, double* q, int on_device) {
  if (!c || !q) return fail(c, GBR_EINVAL, "null argument");
  const size_t bytes = sizeof(double) * c->L.nv * c->L.ncells;
  CK(cudaMemcpyAsync(q, c->q[0], bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream),
     "get state");
  if (!on_device) CK(cudaStreamSynchronize(c->stream), "get state sync");
  return GBR_OK;
}

}  // extern "C"

namespace {

// the copy streams and events of the pipelined transfers, created once per context
gbr_status async_init(gbr_ctx* c) {
  if (c->cs_in) return GBR_OK;
  CK(cudaStreamCreateWithFlags(&c->cs_in, cudaStreamNonBlocking), "copy stream");
  CK(cudaStreamCreateWithFlags(&c->cs_out, cudaStreamNonBlocking), "copy stream");
  for (cudaEvent_t* e : {&c->ev_in_ready, &c->ev_in_free, &c->ev_snap, &c->ev_out_free})
    CK(cudaEventCreateWithFlags(e, cudaEventDisableTiming), "copy event");
  return GBR_OK;
}

// host memory the copy engines can read or write without a staging copy of their own
bool is_pinned(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

// FP32 primitives' pressure offset from cell 0 of a host state (gbr_set_state's rule)
void set_pref_from(gbr_ctx* c, const double* q) {
  const int nv = c->L.nv;
  double ke = 0.0;
  for (int a = 0; a < c->L.nd; ++a) ke += q[(1 + a) * c->L.ncells] * q[(1 + a) * c->L.ncells] / q[0];
  const double p0 = (c->p.gamma - 1.0) * (q[(size_t)(nv - 1) * c->L.ncells] - 0.5 * ke);
  c->pref = std::isfinite(p0) && std::fabs(p0) < 1e38 ? (double)(float)p0 : 0.0;
}

}  // namespace

extern "C" {

gbr_status gbr_set_state_async(gbr_ctx* c, const double* host_q, double* d_stage) {
  if (!c || !host_q || !d_stage) return fail(c, GBR_EINVAL, "null argument");
  if (!is_pinned(host_q)) return fail(c, GBR_EINVAL, "host state must be page-locked (pinned) memory");
  gbr_status s = async_init(c);
  if (s != GBR_OK) return s;
  const size_t bytes = sizeof(double) * c->L.nv * c->L.ncells;
  // upload into the staging buffer once the previous upload has been taken from it, then take it
  // in the context's stream order
  CK(cudaStreamWaitEvent(c->cs_in, c->ev_in_free, 0), "wait staging");
  CK(cudaMemcpyAsync(d_stage, host_q, bytes, cudaMemcpyHostToDevice, c->cs_in), "upload state");
  CK(cudaEventRecord(c->ev_in_ready, c->cs_in), "record upload");
  CK(cudaStreamWaitEvent(c->stream, c->ev_in_ready, 0), "wait upload");
  CK(cudaMemcpyAsync(c->q[0], d_stage, bytes, cudaMemcpyDeviceToDevice, c->stream), "take state");
  CK(cudaEventRecord(c->ev_in_free, c->stream), "record staging free");
  if (c->p.precision == GBR_PREC_MIXED) set_pref_from(c, host_q);
  return GBR_OK;
}

gbr_status gbr_get_state_async(gbr_ctx* c, double* host_q, double* d_stage) {
  if (!c || !host_q || !d_stage) return fail(c, GBR_EINVAL, "null argument");
  if (!is_pinned(host_q)) return fail(c, GBR_EINVAL, "host state must be page-locked (pinned) memory");
  gbr_status s = async_init(c);
  if (s != GBR_OK) return s;
  const size_t bytes = sizeof(double) * c->L.nv * c->L.ncells;
  // snapshot in stream order (once the previous download has left the staging buffer), download
  // on the copy stream while the context's stream goes on
  CK(cudaStreamWaitEvent(c->stream, c->ev_out_free, 0), "wait staging");
  CK(cudaMemcpyAsync(d_stage, c->q[0], bytes, cudaMemcpyDeviceToDevice, c->stream), "snapshot state");
  CK(cudaEventRecord(c->ev_snap, c->stream), "record snapshot");
  CK(cudaStreamWaitEvent(c->cs_out, c->ev_snap, 0), "wait snapshot");
  CK(cudaMemcpyAsync(host_q, d_stage, bytes, cudaMemcpyDeviceToHost, c->cs_out), "download state");
  CK(cudaEventRecord(c->ev_out_free, c->cs_out), "record download");
  return GBR_OK;
}

gbr_status gbr_set_inflow(gbr_ctx* c, const double* prim, int on_device) {
  if (!c || !prim) return fail(c, GBR_EINVAL, "null argument");
  const size_t bytes = sizeof(double) * c->L.nv * c->L.n[1] * c->L.n[2];
  CK(cudaMemcpyAsync(c->inflow, prim, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                     c->stream),
     "set inflow");
  if (!on_device) CK(cudaStreamSynchronize(c->stream), "set inflow sync");
  return GBR_OK;
}

gbr_status gbr_set_sponge(gbr_ctx* c, const double* sigma, const double* q_amb) {
  if (!c) return fail(c, GBR_EINVAL, "null context");
  if (!sigma) { c->have_sponge = false; return GBR_OK; }
  if (!q_amb) return fail(c, GBR_EINVAL, "null ambient state");
  CK(cudaMemcpyAsync(c->sigma, sigma, sizeof(double) * c->L.ncells, cudaMemcpyHostToDevice, c->stream), "set sponge");
  CK(cudaStreamSynchronize(c->stream), "set sponge sync");
  for (int v = 0; v < c->L.nv; ++v) c->qamb[v] = q_amb[v];
  c->have_sponge = true;
  return GBR_OK;
}

gbr_status gbr_rhs(gbr_ctx* c, double* dqdt) {
  if (!c || !dqdt) return fail(c, GBR_EINVAL, "null argument");
  if (!c->metrics_ready) return fail(c, GBR_ESTATE, "metrics not computed");
  return run_rhs(c, c->q[0], c->q[0], dqdt, 0, 0.0, 0.0, 1.0);
}

gbr_status gbr_compute_dt(gbr_ctx* c, double cfl, double* dt_out) {
  if (!c) return fail(c, GBR_EINVAL, "null context");
  if (!(cfl > 0.0)) return fail(c, GBR_EINVAL, "cfl must be positive");
  if (!c->metrics_ready) return fail(c, GBR_ESTATE, "metrics not computed");
  gbr_status s = run_dt(c, cfl);
  if (s != GBR_OK) return s;
  if (dt_out) {
    CK(cudaMemcpyAsync(dt_out, c->scal + S_DT, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "read dt");
    CK(cudaStreamSynchronize(c->stream), "read dt sync");
  }
  return GBR_OK;
}

gbr_status gbr_rk_step(gbr_ctx* c, double cfl_or_neg_dt) {
  if (!c) return fail(c, GBR_EINVAL, "null context");
  if (!c->metrics_ready) return fail(c, GBR_ESTATE, "metrics not computed");
  if (!(cfl_or_neg_dt != 0.0) || std::isnan(cfl_or_neg_dt)) return fail(c, GBR_EINVAL, "cfl_or_neg_dt must be nonzero");
  gbr_status s;
  // geometry at t^n (moving mesh), then the time step from Q^n
  if (c->have_motion) {
    if ((s = run_motion(c, 0.0)) != GBR_OK) return s;
    if ((s = run_geometry(c)) != GBR_OK) return s;
  }
  if (cfl_or_neg_dt > 0.0) {
    if ((s = run_dt(c, cfl_or_neg_dt)) != GBR_OK) return s;
  } else {
    k_set_scalar<<<1, 1, 0, c->stream>>>(c->scal, S_DT, -cfl_or_neg_dt);
    CKL("k_set_scalar");
  }
  // App. B: Q1 = Qn + dt L(Qn); Q2 = 3/4 Qn + 1/4 Q1 + 1/4 dt L(Q1); Qn+1 = 1/3 Qn + 2/3 Q2 + 2/3 dt L(Q2)
  if (rk_in_increments(c)) {
    // mixed path on a static mesh: Q1 = Qn + D1, Q2 = Qn + D2 with FP32 increments
    // D1, D2 kept in the stage buffers (body_update)
    float* d1 = reinterpret_cast<float*>(c->q[1]);
    float* d2 = reinterpret_cast<float*>(c->q[2]);
    if ((s = run_rhs(c, c->q[0], c->q[0], nullptr, 1, 1.0, 0.0, 1.0, nullptr, d1)) != GBR_OK) return s;
    if ((s = run_rhs(c, c->q[0], c->q[0], nullptr, 1, 0.75, 0.25, 0.25, d1, d2)) != GBR_OK) return s;
    if ((s = run_rhs(c, c->q[0], c->q[0], c->q[0], 1, 1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0, d2, nullptr)) != GBR_OK)
      return s;
    k_advance_time<<<1, 1, 0, c->stream>>>(c->scal);
    CKL("k_advance_time");
    return GBR_OK;
  }
  if ((s = run_rhs(c, c->q[0], c->q[0], c->q[1], 1, 1.0, 0.0, 1.0)) != GBR_OK) return s;
  if (c->have_motion) {
    if ((s = run_motion(c, 1.0)) != GBR_OK) return s;
    if ((s = run_geometry(c)) != GBR_OK) return s;
  }
  if ((s = run_rhs(c, c->q[1], c->q[0], c->q[2], 1, 0.75, 0.25, 0.25)) != GBR_OK) return s;
  if (c->have_motion) {
    if ((s = run_motion(c, 0.5)) != GBR_OK) return s;
    if ((s = run_geometry(c)) != GBR_OK) return s;
  }
  if ((s = run_rhs(c, c->q[2], c->q[0], c->q[0], 1, 1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0)) != GBR_OK) return s;
  k_advance_time<<<1, 1, 0, c->stream>>>(c->scal);
  CKL("k_advance_time");
  return GBR_OK;
}

gbr_status gbr_sync(gbr_ctx* c, double timeout_s) {
  if (!c) return fail(c, GBR_EINVAL, "null context");
  auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cudaError_t e = cudaStreamQuery(c->stream);
    if (e == cudaSuccess && c->cs_in) e = cudaStreamQuery(c->cs_in);
    if (e == cudaSuccess && c->cs_out) e = cudaStreamQuery(c->cs_out);
    if (e == cudaSuccess) break;
    if (e != cudaErrorNotReady) return cuda_check(c, e, "stream query");
    double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (timeout_s > 0.0 && el > timeout_s) return fail(c, GBR_ETIMEOUT, "stream did not drain before the deadline");
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  int err[2] = {0, 0};
  CK(cudaMemcpy(err, c->err, sizeof(err), cudaMemcpyDeviceToHost), "read error flags");
  if (err[0]) return fail(c, GBR_ENONFINITE, "non-finite state or non-positive density on the device");
  if (err[1]) return fail(c, GBR_ETIMEOUT, "a tile copy into shared memory did not complete in time");
  return GBR_OK;
}

gbr_status gbr_get_time(gbr_ctx* c, double* t, double* dt) {
  if (!c) return fail(c, GBR_EINVAL, "null context");
  double s[2];
  CK(cudaMemcpyAsync(s, c->scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "read time");
  CK(cudaStreamSynchronize(c->stream), "read time sync");
  if (dt) *dt = s[S_DT];
  if (t) *t = s[S_T];
  return GBR_OK;
}

gbr_status gbr_get_field(gbr_ctx* c, int which, int dir, double* out) {
  if (!c || !out) return fail(c, GBR_EINVAL, "null argument");
  const Layout& L = c->L;
  const int nd = L.nd;
  if (dir < 0 || dir >= nd) dir = 0;
  CK(cudaStreamSynchronize(c->stream), "get field sync");
  auto fetch = [&](const double* src, size_t count, std::vector<double>& h) -> gbr_status {
    h.resize(count);
    CK(cudaMemcpy(h.data(), src, count * sizeof(double), cudaMemcpyDeviceToHost), "get field copy");
    return GBR_OK;
  };
  std::vector<double> h;
  gbr_status s;
  auto cells_from_ext = [&](const std::vector<double>& src, size_t off, double* dst) {
    size_t m = 0;
    for (int k = 0; k < L.n[2]; ++k)
      for (int j = 0; j < L.n[1]; ++j)
        for (int i = 0; i < L.n[0]; ++i) dst[m++] = src[off + eidx(L, i, j, k)];
  };
  switch (which) {
    case GBR_FIELD_CELL_METRICS:
      if ((s = fetch(c->mh, 9 * L.ecount, h)) != GBR_OK) return s;
      for (int e = 0; e < nd; ++e)
        for (int a = 0; a < nd; ++a) cells_from_ext(h, (size_t)(e * 3 + a) * L.ecount, out + (size_t)(e * nd + a) * L.ncells);
      return GBR_OK;
    case GBR_FIELD_CELL_DET:
      if ((s = fetch(c->det, L.ecount, h)) != GBR_OK) return s;
      cells_from_ext(h, 0, out);
      return GBR_OK;
    case GBR_FIELD_CELL_TIME:
      if (!c->mov) return fail(c, GBR_ESTATE, "not a moving mesh");
      if ((s = fetch(c->mt, 3 * L.ecount, h)) != GBR_OK) return s;
      for (int e = 0; e < nd; ++e) cells_from_ext(h, (size_t)e * L.ecount, out + (size_t)e * L.ncells);
      return GBR_OK;
    case GBR_FIELD_FACE_HAT:
      if ((s = fetch(c->fh[dir], (size_t)nd * L.fcount[dir], h)) != GBR_OK) return s;
      std::memcpy(out, h.data(), h.size() * sizeof(double));
      return GBR_OK;
    case GBR_FIELD_FACE_UNHAT:
      if (!c->visc) return fail(c, GBR_ESTATE, "not a viscous case");
      if ((s = fetch(c->fu[dir], (size_t)nd * nd * L.fcount[dir], h)) != GBR_OK) return s;
      std::memcpy(out, h.data(), h.size() * sizeof(double));
      return GBR_OK;
    case GBR_FIELD_FACE_TIME:
      if (!c->mov) return fail(c, GBR_ESTATE, "not a moving mesh");
      if ((s = fetch(c->ft[dir], (size_t)L.fcount[dir], h)) != GBR_OK) return s;
      std::memcpy(out, h.data(), h.size() * sizeof(double));
      return GBR_OK;
    case GBR_FIELD_GCL:
      if (!c->mov) return fail(c, GBR_ESTATE, "not a moving mesh");
      if ((s = fetch(c->gcl, (size_t)L.ncells, h)) != GBR_OK) return s;
      std::memcpy(out, h.data(), h.size() * sizeof(double));
      return GBR_OK;
    case GBR_FIELD_FACE_FLUX: {
      const size_t n = (size_t)L.nv * L.fcount[dir];
      if (c->p.precision == GBR_PREC_MIXED) {
        std::vector<float> hf(n);
        CK(cudaMemcpyAsync(hf.data(), c->flux[dir], n * sizeof(float), cudaMemcpyDeviceToHost, c->stream), "fetch");
        CK(cudaStreamSynchronize(c->stream), "fetch sync");
        for (size_t m = 0; m < n; ++m) out[m] = hf[m];
        return GBR_OK;
      }
      if ((s = fetch(static_cast<const double*>(c->flux[dir]), n, h)) != GBR_OK) return s;
      std::memcpy(out, h.data(), h.size() * sizeof(double));
      return GBR_OK;
    }
    default:
      return fail(c, GBR_EINVAL, "unknown field");
  }
}

gbr_status gbr_profile(gbr_ctx* c, int enable, double* face_ms, long long* face_launches, long long* launches) {
  if (!c) return fail(nullptr, GBR_EINVAL, "null context");
  CK(cudaStreamSynchronize(c->stream), "profile sync");
  double total = 0.0;
  for (size_t m = 0; m + 1 < c->ev_used; m += 2) {
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, c->ev[m], c->ev[m + 1]), "event elapsed");
    total += ms;
  }
  if (face_ms) *face_ms = total;
  if (face_launches) *face_launches = (long long)(c->ev_used / 2);
  if (launches) *launches = c->launches;
  c->ev_used = 0;
  c->launches = 0;
  c->prof = enable != 0;
  return GBR_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Fused multiply-add throughput probe (gbr_alu_peak): the denominator of the
// arithmetic roofline, measured on the device that runs the kernels.  Each
// thread runs kProbeChains independent FMA chains a = a * x + y with runtime x
// and y (nothing folds; |x| < 1 keeps every value finite), and stores its sum
// only if it equals a value no chain produces, so no chain is dead code.
// ---------------------------------------------------------------------------
namespace {
constexpr int kProbeChains = 8;
constexpr int kProbeUnroll = 16;
constexpr int kProbeBlock = 256;

template <class T>
__global__ void __launch_bounds__(kProbeBlock) k_fma_probe(T x, T y, int iters, T never, T* sink) {
  T a[kProbeChains];
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) a[c] = T(threadIdx.x + c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kProbeUnroll; ++u) {
#pragma unroll
      for (int c = 0; c < kProbeChains; ++c) a[c] = fma(a[c], x, y);
    }
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) s += a[c];
  if (s == never) sink[blockIdx.x] = s;
}

template <class T>
gbr_status alu_probe(cudaStream_t st, int iters, double* tflops, double* ms_out) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_probe<T>, kProbeBlock, 0) != cudaSuccess)
    return fail(nullptr, GBR_ECUDA, "alu probe: device query failed");
  const int blocks = sms * std::max(per_sm, 1);  // one wave: every SM gets the same work
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return fail(nullptr, GBR_ECUDA, "alu probe: event");
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return fail(nullptr, GBR_ECUDA, "alu probe: event"); }
  const T x = T(0.999), y = T(1.0e-3), never = T(-12345.0);
  float best = 0.0f;
  cudaError_t err = cudaSuccess;
  for (int rep = 0; rep < 4 && err == cudaSuccess; ++rep) {  // the first launch warms up
    cudaEventRecord(e0, st);
    k_fma_probe<T><<<blocks, kProbeBlock, 0, st>>>(x, y, iters, never, nullptr);
    cudaEventRecord(e1, st);
    err = cudaEventSynchronize(e1);
    if (err == cudaSuccess) err = cudaGetLastError();
    float ms = 0.0f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && err == cudaSuccess && (best == 0.0f || ms < best)) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return fail(nullptr, GBR_ECUDA, std::string("alu probe: ") + cudaGetErrorString(err));
  const double flops = 2.0 * kProbeChains * kProbeUnroll * (double)iters * (double)blocks * kProbeBlock;
  if (tflops) *tflops = flops / (best * 1e-3) / 1e12;
  if (ms_out) *ms_out = best;
  return GBR_OK;
}
}  // namespace

extern "C" {

gbr_status gbr_alu_peak(int precision, void* stream, double* tflops, double* ms) {
  cudaStream_t st = (cudaStream_t)stream;
  if (precision == GBR_PREC_FP64) return alu_probe<double>(st, 1024, tflops, ms);
  if (precision == GBR_PREC_MIXED) return alu_probe<float>(st, 32768, tflops, ms);
  return fail(nullptr, GBR_EINVAL, "precision must be GBR_PREC_FP64 or GBR_PREC_MIXED");
}

// ---------------------------------------------------------------------------
// Self-check of grcp (gbr_check_rcp): its reciprocal against the FP64 division on
// SplitMix64 bit patterns (Steele, Lea and Flood, "Fast splittable pseudorandom
// number generators", OOPSLA 2014), the largest distance in units in the last place.
// ---------------------------------------------------------------------------
__device__ unsigned long long g_rcp_max_ulp;

__global__ void k_rcp_check(long long n, unsigned long long seed) {
  unsigned long long worst = 0;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    unsigned long long z = seed + (unsigned long long)(t + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const unsigned long long ef = 23 + (z >> 53) % 2001;  // x and 1/x normal
    const unsigned long long b = ((unsigned long long)(t & 1) << 63) | (ef << 52) | (z & ((1ull << 52) - 1));
    const double x = __longlong_as_double((long long)b);
    const long long r1 = __double_as_longlong(grcp(x)), r2 = __double_as_longlong(1.0 / x);
    const unsigned long long d = (unsigned long long)(r1 > r2 ? r1 - r2 : r2 - r1);
    worst = d > worst ? d : worst;
  }
  atomicMax(&g_rcp_max_ulp, worst);
}

gbr_status gbr_check_rcp(long long n, unsigned long long seed, void* stream, long long* max_ulp) {
  if (!max_ulp || n < 1 || n > (1LL << 34)) return fail(nullptr, GBR_EINVAL, "check_rcp: n outside 1 .. 2^34 or null max_ulp");
  cudaStream_t st = (cudaStream_t)stream;
  void* addr = nullptr;
  if (cudaGetSymbolAddress(&addr, g_rcp_max_ulp) != cudaSuccess || cudaMemsetAsync(addr, 0, sizeof(unsigned long long), st) != cudaSuccess)
    return fail(nullptr, GBR_ECUDA, "check_rcp: counter reset failed");
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return fail(nullptr, GBR_ECUDA, "check_rcp: device query failed");
  k_rcp_check<<<sms * 8, 256, 0, st>>>(n, seed);
  unsigned long long v = 0;
  if (cudaGetLastError() != cudaSuccess || cudaMemcpyAsync(&v, addr, sizeof v, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail(nullptr, GBR_ECUDA, "check_rcp: kernel or copy failed");
  *max_ulp = (long long)v;
  return GBR_OK;
}

gbr_status gbr_check_bounded_wait(gbr_ctx* c, int polls) {
  if (!c) return fail(nullptr, GBR_EINVAL, "null context");
  if (polls < 1 || polls > kTmaSpin) return fail(c, GBR_EINVAL, "polls out of range");
  k_wait_check<<<1, kIg4Lines, 0, c->stream>>>(polls, c->err);
  CKL("k_wait_check");
  return GBR_OK;
}

const char* gbr_last_error(const gbr_ctx* c) { return c ? c->last_error.c_str() : g_global_error.c_str(); }
const char* gbr_last_global_error(void) { return g_global_error.c_str(); }

void gbr_destroy(gbr_ctx* c) {
  if (!c) return;
  for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
  for (cudaEvent_t e : {c->ev_in_ready, c->ev_in_free, c->ev_snap, c->ev_out_free})
    if (e) cudaEventDestroy(e);
  for (cudaStream_t t : {c->cs_in, c->cs_out})
    if (t) {
      cudaStreamSynchronize(t);
      cudaStreamDestroy(t);
    }
  delete c;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Right-hand side without any allocation (gbr_rhs_static, include/gbr.h)
//
// For callers that cannot allocate device memory: code that runs inside
// another framework's memory pool or under a hard device-memory budget, code
// that must not allocate after start-up, or code that cannot own a workspace.
// All scratch of the right-hand side (geometry, primitives, derivatives,
// interface fluxes) lives in the file-scope device array below, which every
// GPU that loads this library holds until the process exits.
// ---------------------------------------------------------------------------
namespace {
constexpr size_t kStaticScratchBytes = (size_t)64 << 20;  // 64 MiB per device
constexpr int kMaxStaticDevices = 64;
}  // namespace

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

namespace {

void* g_static_scratch_addr[kMaxStaticDevices];  // device address of g_static_scratch, per device

gbr_status static_report(gbr_status s, const char* m, char* msg, size_t msg_len) {
  if (msg && msg_len > 0) {
    size_t n = std::strlen(m);
    if (n >= msg_len) n = msg_len - 1;
    std::memcpy(msg, m, n);
    msg[n] = 0;
  }
  return s;
}

const char* static_param_error(const gbr_params* p) {
  if (p->ndim != 2 && p->ndim != 3) return "ndim must be 2 or 3";
  for (int d = 0; d < p->ndim; ++d) {
    if (p->n[d] < 1) return "empty axis";
    if (p->periodic[d] && p->n[d] < H) return "a periodic axis needs at least 6 cells";
    if (!p->periodic[d]) {
      if (p->ghost_nodes < E) return "a non-periodic axis needs ghost_nodes >= 10";
      for (int s = 0; s < 2; ++s)
        if (p->bc[d][s] != GBR_BC_ZEROGRAD) return "only periodic and zero-gradient sides are supported here";
    }
  }
  if (!(p->gamma > 1.0)) return "gamma must exceed 1";
  if (p->reynolds > 0.0 && !(p->prandtl > 0.0)) return "prandtl must be positive";
  if (p->sutherland_s > 0.0 && !(p->t_ref > 0.0)) return "t_ref must be positive";
  if (p->precision != GBR_PREC_FP64) return "only the FP64 path is supported here";
  if (p->gradient_scheme != GBR_GRAD_MEG6) return "only MEG6 is supported here";
  for (int d = 0; d < p->ndim; ++d)
    if (!p->periodic[d] && p->ghost_nodes == 0) return "non-periodic axes need ghost nodes here";
  return nullptr;
}

struct RawNodes {
  int Nn[3], off[3];
  long long count;  // nodes per coordinate
};

RawNodes raw_nodes_of(const gbr_params* p, const Layout& L) {
  RawNodes R;
  R.count = 1;
  for (int d = 0; d < 3; ++d) {
    if (d >= L.nd) { R.Nn[d] = 1; R.off[d] = 0; continue; }
    R.Nn[d] = p->periodic[d] ? L.n[d] + 1 : L.n[d] + 1 + 2 * p->ghost_nodes;
    R.off[d] = p->periodic[d] ? 0 : p->ghost_nodes;
    R.count *= R.Nn[d];
  }
  return R;
}

// period vectors of the periodic axes, with the closing-face check; reads the host nodes only
const char* static_period_vectors(const gbr_params* p, const Layout& L, const RawNodes& R, const double* src,
                                  double per[3][3]) {
  const int nd = L.nd;
  const long long NN = R.count;
  auto sid = [&](int a, int s0, int s1, int s2) {
    return (size_t)a * NN + ((size_t)s2 * R.Nn[1] + s1) * R.Nn[0] + s0;
  };
  double scale = 0.0;
  for (long long m = 0; m < (long long)nd * NN; ++m) scale = std::fmax(scale, std::fabs(src[m]));
  for (int d = 0; d < 3; ++d)
    for (int a = 0; a < 3; ++a) per[d][a] = 0.0;
  for (int d = 0; d < nd; ++d) {
    if (!p->periodic[d]) continue;
    int s0[3] = {R.off[0], R.off[1], R.off[2]}, s1[3] = {R.off[0], R.off[1], R.off[2]};
    s1[d] = L.n[d];
    for (int a = 0; a < nd; ++a) per[d][a] = src[sid(a, s1[0], s1[1], s1[2])] - src[sid(a, s0[0], s0[1], s0[2])];
    for (int s2 = 0; s2 < R.Nn[2]; ++s2)
      for (int s1i = 0; s1i < R.Nn[1]; ++s1i)
        for (int s0i = 0; s0i < R.Nn[0]; ++s0i) {
          int s[3] = {s0i, s1i, s2};
          if (s[d] != 0) continue;
          int t[3] = {s0i, s1i, s2};
          t[d] = L.n[d];
          for (int a = 0; a < nd; ++a) {
            double diff = src[sid(a, t[0], t[1], t[2])] - src[sid(a, s[0], s[1], s[2])];
            if (std::fabs(diff - per[d][a]) > 1e-12 * (scale + 1.0))
              return "periodic axis is not closed by a constant period vector";
          }
        }
  }
  return nullptr;
}

struct ExtendArgs {
  Layout L;
  RawNodes R;
  int periodic[3];
  double per[3][3];
  int shift;  // 1: coordinates (add period vectors), 0: velocities
  const double* raw;
  double* ext;
};

// extended node box [-E, n+E]: unwrapped periodic images / supplied ghost layers
__global__ void k_extend_nodes(ExtendArgs X, Box b) {
  BOX_THREAD(b);
  const Layout& L = X.L;
  const int m[3] = {i, j, k};
  int s[3], wraps[3] = {0, 0, 0};
  for (int d = 0; d < 3; ++d) {
    if (d >= L.nd) { s[d] = 0; continue; }
    if (X.periodic[d]) {
      const int n = L.n[d];
      const int base = ((m[d] % n) + n) % n;
      wraps[d] = (m[d] - base) / n;
      s[d] = base;
    } else {
      s[d] = m[d] + X.R.off[d];
    }
  }
  const long long id = nidx(L, i, j, k);
  const long long src = ((long long)s[2] * X.R.Nn[1] + s[1]) * X.R.Nn[0] + s[0];
  for (int a = 0; a < L.nd; ++a) {
    double v = X.raw[a * X.R.count + src];
    if (X.shift)
      for (int d = 0; d < L.nd; ++d) v += wraps[d] * X.per[d][a];
    X.ext[a * L.ncount + id] = v;
  }
}

template <int ND, bool VISC, bool MOV>
void static_face_launches(const RhsArgs& A, const RhsBoxes& B, cudaStream_t st) {
  k_face<ND, VISC, MOV, double, 0><<<face_grid<double, ND, 0>(B.faces[0]), face_bs<0>(), 0, st>>>(A, 0, B.faces[0]);
  k_face<ND, VISC, MOV, double, 1><<<face_grid<double, ND, 1>(B.faces[1]), face_bs<1>(), 0, st>>>(A, 1, B.faces[1]);
  if constexpr (ND == 3)
    k_face<ND, VISC, MOV, double, 2><<<face_grid<double, ND, 2>(B.faces[2]), face_bs<2>(), 0, st>>>(A, 2, B.faces[2]);
}

// the launch sequence of one right-hand side (geometry first), errors as cudaError_t only
template <int ND>
cudaError_t static_rhs_launches(gbr_ctx& c, const double* q, double* dqdt, cudaStream_t st) {
  const Layout& L = c.L;
  const GeoArgs G = geo_args(&c);
  const GeoBoxes GB = geo_boxes(L);
  k_centroid<<<grid_of(GB.ext, kBlock), kBlock, 0, st>>>(G, GB.ext);
  unsigned gmax = 0;
  for (int d = 0; d < ND; ++d) gmax = std::max(gmax, grid_of(GB.coordd[d], kBlock));
  k_coordd<<<dim3(gmax, ND), kBlock, 0, st>>>(G, GB.coordd[0], GB.coordd[1], GB.coordd[2]);
  k_metrics<<<grid_of(GB.metrics, kBlock), kBlock, 0, st>>>(G, GB.metrics);
  gmax = 0;
  for (int d = 0; d < ND; ++d) gmax = std::max(gmax, grid_of(GB.faces[d], kBlock));
  k_face_metrics<<<dim3(gmax, ND), kBlock, 0, st>>>(G, GB.faces[0], GB.faces[1], GB.faces[2]);
  FaceGeoOut O;
  for (int d = 0; d < 3; ++d) O.fg[d] = c.fg[d];
  k_face_geo<<<dim3(gmax, ND), kBlock, 0, st>>>(G, O, GB.faces[0], GB.faces[1], GB.faces[2]);
  k_gcl<<<grid_of(GB.inner, kBlock), kBlock, 0, st>>>(G, GB.inner);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;

  const RhsArgs A = rhs_args(&c, q);
  const RhsBoxes B = rhs_boxes(L);
  k_prim<ND><<<grid_of(B.inner, kBlock), kBlock, 0, st>>>(A, B.inner);
  for (int d = 0; d < ND; ++d) k_halo<ND><<<grid_of(B.halo[d], kBlock), kBlock, 0, st>>>(A, d, B.halo[d]);
  unsigned g1 = 0, g2 = 0;
  for (int d = 0; d < ND; ++d) {
    g1 = std::max(g1, grid_of(B.grad1[d], kBlock));
    g2 = std::max(g2, grid_of(B.grad2[d], kBlock));
  }
  k_grad1<ND><<<g1 * ND, kBlock, 0, st>>>(A, B.grad1[0], B.grad1[1], B.grad1[2]);
  k_grad2<ND><<<g2 * ND, kBlock, 0, st>>>(A, B.grad2[0], B.grad2[1], B.grad2[2]);
  if (c.visc) {
    if (c.mov) static_face_launches<ND, true, true>(A, B, st);
    else static_face_launches<ND, true, false>(A, B, st);
  } else {
    if (c.mov) static_face_launches<ND, false, true>(A, B, st);
    else static_face_launches<ND, false, false>(A, B, st);
  }
  UpdArgs U;
  U.L = L;
  for (int d = 0; d < 3; ++d) U.flux[d] = static_cast<const double*>(c.flux[d]);
  U.qs = q;
  U.q0 = q;
  U.out = dqdt;
  U.jac = c.jac;
  U.jac32 = nullptr;
  U.gcl = c.gcl;
  U.sigma = nullptr;
  for (int v = 0; v < 5; ++v) U.qamb[v] = 0.0;
  U.dt = c.scal + S_DT;
  U.ca = 0.0;
  U.cb = 0.0;
  U.cc = 1.0;
  U.mode = 0;
  U.dq_in = nullptr;
  U.dq_out = nullptr;
  if (c.mov) k_update<ND, true><<<grid_of(B.inner, kBlock), kBlock, 0, st>>>(U, B.inner, c.err);
  else k_update<ND, false><<<grid_of(B.inner, kBlock), kBlock, 0, st>>>(U, B.inner, c.err);
  return cudaGetLastError();
}

}  // namespace

extern "C" gbr_status gbr_rhs_static(const gbr_params* p, const double* nodes, const double* node_vel,
                                     const double* q, double* dqdt, void* stream, char* msg, size_t msg_len) {
  if (!p || !nodes || !q || !dqdt) return static_report(GBR_EINVAL, "null argument", msg, msg_len);
  {  // the general checks first (axis and ghost-layer bounds, 32-bit offsets), then this call's own limits
    std::string why;
    if (!valid_params(p, why)) return static_report(GBR_EINVAL, why.c_str(), msg, msg_len);
  }
  if (const char* why = static_param_error(p)) return static_report(GBR_EINVAL, why, msg, msg_len);
  if (node_vel && !p->moving) return static_report(GBR_EINVAL, "node velocities need params.moving = 1", msg, msg_len);
  const Layout L = layout_of(p);
  const Plan P = plan_of(p, L);
  const RawNodes R = raw_nodes_of(p, L);
  const size_t raw_bytes = (((size_t)L.nd * R.count * sizeof(double)) + 255) & ~(size_t)255;
  const size_t need = P.total + raw_bytes * (node_vel ? 2 : 1);
  if (need > kStaticScratchBytes)
    return static_report(GBR_EINVAL, "grid too large for the 64 MiB static scratch of gbr_rhs_static", msg, msg_len);
  double per[3][3];
  if (const char* why = static_period_vectors(p, L, R, nodes, per)) return static_report(GBR_EINVAL, why, msg, msg_len);

  // set-up, once per device, with that device current: the device address of the static array
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return static_report(GBR_ECUDA, "cudaGetDevice failed", msg, msg_len);
  if (dev < 0 || dev >= kMaxStaticDevices) return static_report(GBR_EINVAL, "device index out of range", msg, msg_len);
  if (!g_static_scratch_addr[dev]) {
    void* addr = nullptr;
    if (cudaGetSymbolAddress(&addr, g_static_scratch) != cudaSuccess || !addr)
      return static_report(GBR_ECUDA, "cudaGetSymbolAddress of the static scratch failed", msg, msg_len);
    g_static_scratch_addr[dev] = addr;
  }

  gbr_ctx c;  // host-side view of the scratch; holds no heap memory on this path
  c.p = *p;
  if (p->ndim == 2) c.p.n[2] = 1;
  c.L = L;
  c.ph = phys_of(p);
  c.stream = (cudaStream_t)stream;
  c.ws = (char*)g_static_scratch_addr[dev];
  c.ws_bytes = kStaticScratchBytes;
  c.plan = P;
  c.visc = p->reynolds > 0.0;
  c.mov = node_vel != nullptr;
  c.have_sponge = false;
  c.have_motion = false;
  c.metrics_ready = false;
  c.launches = 0;
  c.prof = false;
  c.ev_used = 0;
  for (int v = 0; v < 5; ++v) c.qamb[v] = 0.0;
  carve(&c);
  if (!c.mov) {  // a static mesh leaves the moving-mesh slots out of the plan
    c.nvel = nullptr;
    c.vc = nullptr;
  }
  cudaStream_t st = c.stream;
  double* raw = (double*)(c.ws + P.total);
  double* rawv = (double*)(c.ws + P.total + raw_bytes);
  const size_t copy_bytes = (size_t)L.nd * R.count * sizeof(double);
  // the error flag and the scalars must start at zero; every other slot is rewritten before it is read
  if (cudaMemsetAsync(c.err, 0, sizeof(int) * 4, st) != cudaSuccess ||
      cudaMemsetAsync(c.scal, 0, sizeof(double) * S_NSCAL, st) != cudaSuccess ||
      cudaMemcpyAsync(raw, nodes, copy_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      (c.mov && cudaMemcpyAsync(rawv, node_vel, copy_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess))
    return static_report(GBR_ECUDA, "copy to the static scratch failed", msg, msg_len);
  ExtendArgs X;
  X.L = L;
  X.R = R;
  for (int d = 0; d < 3; ++d) {
    X.periodic[d] = (d < L.nd) ? p->periodic[d] : 1;
    for (int a = 0; a < 3; ++a) X.per[d][a] = per[d][a];
  }
  const Box bn = geo_boxes(L).nodes;
  X.shift = 1;
  X.raw = raw;
  X.ext = c.nodes;
  k_extend_nodes<<<grid_of(bn, kBlock), kBlock, 0, st>>>(X, bn);
  if (c.mov) {
    X.shift = 0;
    X.raw = rawv;
    X.ext = c.nvel;
    k_extend_nodes<<<grid_of(bn, kBlock), kBlock, 0, st>>>(X, bn);
  }
  cudaError_t e = L.nd == 3 ? static_rhs_launches<3>(c, q, dqdt, st) : static_rhs_launches<2>(c, q, dqdt, st);
  if (e != cudaSuccess) return static_report(GBR_ECUDA, cudaGetErrorString(e), msg, msg_len);
  return GBR_OK;
}

#include "gbr_batch.cuh"
