// Batched stepping of many contexts and the device-memory arena used to admit them.
//
// Included at the end of gbr.cu (one translation unit: it uses the context
// layout, the launch helpers and the kernel bodies).  Not in the paper, whose
// solver runs one job per GPU; the arithmetic of every member is exactly that of
// gbr_rk_step on the member alone (same bodies, same data, same order).
//
// Design:
// * Members are grouped by kind: (ndim, viscous, precision, moving mesh, gradient
//   scheme).  Per kind, each
//   phase of an SSP-RK3 step is ONE launch over a work list of items
//   (member, sub-box, first block, blocks): the block -> (member, tile) map.
//   Moving-mesh members also recompute their geometry at each stage time (their
//   own motion, metric and GCL launches, in gbr_rk_step's order), and MIG4
//   members solve their IG4 lines with their own launches; the other phases of
//   those kinds are batched as for the rest.
// * Phase kernels are persistent: the grid is the number of co-resident CTAs (or
//   fewer), and CTA b takes the contiguous block range [b*chunk, (b+1)*chunk)
//   of the work list, finding its first item by binary search and walking on.
// * Primitives and all ghost layers are produced by one pass over the padded box
//   (body_prim_halo), so a stage is prim+halo, gradients, interfaces, update.
// * The whole step (time step on the device, three stages, time advance, for
//   every kind) is captured once into a CUDA graph and replayed until the
//   membership changes.
// * Per kind, an autotuner picks the interface kernel's block size (interfaces
//   per tile: 64, 128 or 256) and the gradient sweep (two passes, or one fused
//   pass that recomputes the neighbours' first derivatives) by timing the
//   stage-1 right-hand side of the live members; results are cached per kind and
//   size class (log2 of the kind's cells).

namespace {

// ---------------------------------------------------------------------------
// device tables
// ---------------------------------------------------------------------------
template <class R>
struct BatchJob {
  RhsArgsT<R> A;        // A.q unused: the stage input comes from q[stage]
  UpdArgsT<R> U[4];     // SSP-RK3 stage combinations 0..2; 3: L(Q^n) into Q^(1) (autotuning)
  DtArgs D;
  const double* q[3];   // Q^n, Q^(1), Q^(2) (increment form: Q^n for every stage)
  const float* dq[3];   // increment form: null, D1, D2 (the stage state is q[s] + dq[s])
  Box pad, inner, grad1[3], grad2[3], faces[3];
  double* scal;
  unsigned long long* dtbits;
  int* err;
  double cfl;           // > 0: CFL number; < 0: fixed time step -cfl
  Box g1u;              // WL_G1V members: k_grad1v's box union and tiles_x, tiles_y, zchunk, chunks
  int g1v[4];
};

struct WorkItem {
  int job, sub, first, blocks;  // blocks [first, first + blocks) of the launch cover sub-box `sub` of `job`
};

// WL_G1V: FP32 3D MEG6 members whose rows are 16-byte aligned take their first derivatives by
// k_grad1v's tiles (one item per member: its tiles x chunks x fields), the others cell by cell
// (WL_GRAD1); the fused stage kernel keeps every member on WL_GRAD1
enum { WL_PAD = 0, WL_GRAD1, WL_GRAD2, WL_FACE, WL_INNER, WL_DT, WL_G1V, WL_COUNT };

// Runs f(item, local block) for the contiguous block range of this CTA.  The items may be a
// sub-range of a longer list: `base` is the block offset its first item starts at.
template <class F>
__device__ __forceinline__ void for_work(const WorkItem* items, int n_items, int total, F f, int base = 0) {
  const int chunk = (total + (int)gridDim.x - 1) / (int)gridDim.x;
  const int b0 = (int)blockIdx.x * chunk;
  const int b1 = min(total, b0 + chunk);
  if (b0 >= b1) return;
  int lo = 0, hi = n_items - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (items[mid].first <= b0 + base) lo = mid;
    else hi = mid - 1;
  }
  int m = lo;
  for (int blk = b0 + base; blk < b1 + base; ++blk) {
    while (m + 1 < n_items && blk >= items[m].first + items[m].blocks) ++m;
    f(items[m], blk - items[m].first);
  }
}

// Runs f(item, local block) for block blockIdx.x + base of a list launched with one CTA per work
// block (no loop: the interface kernels keep their registers for the interface)
template <class F>
__device__ __forceinline__ void one_work(const WorkItem* items, int n_items, F f, int base = 0) {
  const int blk = (int)blockIdx.x + base;
  int lo = 0, hi = n_items - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (items[mid].first <= blk) lo = mid;
    else hi = mid - 1;
  }
  f(items[lo], blk - items[lo].first);
}

// the phase kernels' loop: one work block per CTA (GBR_BATCH_ONE, grid = the list's blocks), or
// a persistent range of them per CTA.  One per CTA measured faster for every phase (batch steps of
// twelve 48^3-64^3 TGV jobs / four 96^3, the interface kernels already one per CTA: FP64 18.99 ->
// 18.49 ms / 28.84 -> 28.10 ms, mixed 2.784 -> 2.544 ms): the block scheduler balances the
// uneven members' blocks better than fixed ranges, and no loop state takes registers.
#ifndef GBR_BATCH_ONE
#define GBR_BATCH_ONE 1
#endif
template <class F>
__device__ __forceinline__ void phase_work(const WorkItem* items, int n_items, int total, F f) {
  if constexpr (GBR_BATCH_ONE) {
    if ((int)blockIdx.x < total && n_items > 0) one_work(items, n_items, f);
  } else {
    for_work(items, n_items, total, f);
  }
}

#define BATCH_CELL(BOX)                                                        \
  const long long _t = (long long)lb * blockDim.x + threadIdx.x;              \
  if (_t >= box_size(BOX)) return;                                             \
  int i, j, k;                                                                 \
  box_coord(BOX, _t, i, j, k);

template <int ND, class R>
__global__ void __launch_bounds__(kBlock, kStreamBlocks) kb_prim_halo(const BatchJob<R>* jobs, const WorkItem* items, int n,
                                                        int total, int stage) {
  phase_work(items, n, total, [&](const WorkItem& it, int lb) {
    const BatchJob<R>& J = jobs[it.job];
    BATCH_CELL(J.pad);
    body_prim_halo<ND>(J.A, J.q[stage], J.dq[stage], i, j, k);
  });
}

template <int ND, class R>
__global__ void __launch_bounds__(kBlock) kb_grad1(const BatchJob<R>* jobs, const WorkItem* items, int n, int total) {
  phase_work(items, n, total, [&](const WorkItem& it, int lb) {
    const BatchJob<R>& J = jobs[it.job];
    BATCH_CELL(J.grad1[it.sub]);
    body_grad1<ND>(J.A, it.sub, i, j, k);
  });
}

template <int ND, class R>
__global__ void __launch_bounds__(kBlock) kb_grad2(const BatchJob<R>* jobs, const WorkItem* items, int n, int total) {
  phase_work(items, n, total, [&](const WorkItem& it, int lb) {
    const BatchJob<R>& J = jobs[it.job];
    BATCH_CELL(J.grad2[it.sub]);
    body_grad2<ND>(J.A, it.sub, i, j, k);
  });
}

// fused gradient sweep over the first-derivative box: f' everywhere, f'' where the
// second-derivative box needs it, from f' of the neighbours recomputed in registers
// the tiles of k_grad1v over the WL_G1V items (FP32 3D), one tile per CTA
__global__ void __launch_bounds__(kGVX * kGVY, GBR_G1V_MINB) kb_grad1v(const BatchJob<float>* jobs, const WorkItem* items,
                                                                    int n, int total) {
  __shared__ float4 plane[2][kGVR * kGVW];
  phase_work(items, n, total, [&](const WorkItem& it, int lb) {
    const BatchJob<float>& J = jobs[it.job];
    const int per_field = J.g1v[0] * J.g1v[1] * J.g1v[3];
    grad1v_tile(J.A, J.g1u, J.grad1[0], J.grad1[1], J.grad1[2], J.g1v[0], J.g1v[1], J.g1v[2], lb % per_field,
                lb / per_field, plane);
  });
}

template <int ND, class R>
__global__ void __launch_bounds__(kBlock) kb_grad12(const BatchJob<R>* jobs, const WorkItem* items, int n,
                                                     int total) {
  phase_work(items, n, total, [&](const WorkItem& it, int lb) {
    const BatchJob<R>& J = jobs[it.job];
    BATCH_CELL(J.grad1[it.sub]);
    body_grad12<ND>(J.A, it.sub, J.grad2[it.sub], i, j, k);
  });
}

// As k_face: the limiter's bound work compacted over the block (every thread takes part in
// each work block's barriers); FP32 at 896 threads per SM in 3D (7 blocks of 128, as k_face:
// 72 registers, some spilled, measured faster than 768 or 640 threads without spills on a batch
// of 48^3-64^3 mixed TGV jobs) and 768 in 2D (5 % faster than 896 on 96^2-160^2 vortex jobs),
// FP64 at 512 threads (4 blocks of 128 at 128 registers, as k_face).  Each CTA runs one work
// block (GBR_BATCH_FACE_ONE: grid = the direction's blocks, the item found by a binary search)
// instead of a persistent loop over a range of them: without the loop's state the FP64 kernel
// fits 128 registers without spills (persistent it took 168, 3 blocks per SM, and spilled at
// 128), and the FP32 one spills less.  Batch steps (twelve 48^3-64^3 TGV jobs / four 96^3):
// FP64 20.49 -> 18.98 ms / 30.77 -> 28.84 ms, mixed 3.155 -> 2.788 ms.  The FP64 3D x-sweep takes
// k_face's transposed mapping (-1.0 / -1.2 % per step on those batches).
// DD: the one sweep direction of the launch's items (the per-direction instantiation, as k_face)
#ifndef GBR_BATCH_FACE_FP64_THREADS
#define GBR_BATCH_FACE_FP64_THREADS 512
#endif
#ifndef GBR_BATCH_FACE_ONE
#define GBR_BATCH_FACE_ONE 1
#endif
#ifndef GBR_BATCH_FACE_F32_THREADS_3D
#define GBR_BATCH_FACE_F32_THREADS_3D 896  // 768 (80 registers, no spill): +3 % per mixed batch step
#endif
template <int ND, bool VISC, bool MOV, class R, int BS, int DD>
__global__ void __launch_bounds__(BS, sizeof(R) == 4 ? (ND == 3 ? GBR_BATCH_FACE_F32_THREADS_3D : 768) / BS
                                                     : (BS < GBR_BATCH_FACE_FP64_THREADS ? GBR_BATCH_FACE_FP64_THREADS / BS : 1))
    kb_face(const BatchJob<R>* jobs, const WorkItem* items, int n, int total, int base) {
  __shared__ BoundSlot<ND, R> slots[BS];
  __shared__ int count;
  auto work = [&](auto&& f) {
    if constexpr (GBR_BATCH_FACE_ONE) one_work(items, n, f, base);
    else for_work(items, n, total, f, base);
  };
  work([&](const WorkItem& it, int lb) {
    const BatchJob<R>& J = jobs[it.job];
    bool valid;
    int i = 0, j = 0, k = 0;
    if constexpr (face_xt<R, ND, DD>() > 0) {
      // the transposed x-sweep mapping of k_face (its blocks counted so by build_items)
      valid = face_xt_coord<BS, face_xt<R, ND, DD>()>(J.faces[DD], lb, (int)threadIdx.x, i, j, k);
    } else {
      const long long t = (long long)lb * blockDim.x + threadIdx.x;
      valid = t < box_size(J.faces[DD]);
      if (valid) box_coord(J.faces[DD], t, i, j, k);
    }
    face_block<ND, VISC, MOV, R, DD>(J.A, DD, valid, i, j, k, slots, &count);
  });
}

template <int ND, bool MOV, class R, bool SP>
__global__ void __launch_bounds__(kBlock, kStreamBlocks) kb_update(const BatchJob<R>* jobs, const WorkItem* items, int n, int total,
                                                     int stage) {
  phase_work(items, n, total, [&](const WorkItem& it, int lb) {
    const BatchJob<R>& J = jobs[it.job];
    BATCH_CELL(J.inner);
    if (body_update<ND, MOV, R, SP>(J.U[stage], i, j, k)) atomicOr(J.err, 1);
  });
}

// ---------------------------------------------------------------------------
// One persistent, fused right-hand side per kind and stage: the phases (primitives and ghost
// layers, gradients, interface fluxes, update) of every member run in ONE cooperative launch
// over the block -> (member, tile) work lists, separated by grid-wide barriers.  The launch is
// cooperative, so every CTA is resident and each barrier completes once all CTAs arrive; the
// wait is bounded all the same: a barrier that has not completed after kGridBarSpin polls sets
// the kind's timeout flag (gbr_batch_sync reports GBR_ETIMEOUT) and the CTA goes on.
// ---------------------------------------------------------------------------
constexpr int kGridBarSpin = 1 << 22;
constexpr int kFusedBlock = 128;

struct GridBar {
  unsigned* count;  // arrivals at the current barrier
  unsigned* gen;    // completed barriers
  int* timeout;
};

__device__ __forceinline__ void grid_barrier(const GridBar& G, int spins = kGridBarSpin) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vg = G.gen;
    const unsigned g = *vg;
    __threadfence();
    if (atomicAdd(G.count, 1u) == gridDim.x - 1) {
      atomicExch(G.count, 0u);
      __threadfence();
      atomicAdd(G.gen, 1u);
    } else {
      int it = 0;
      while (*vg == g && it < spins) {
        __nanosleep(200);
        ++it;
      }
      if (it >= spins) atomicOr(G.timeout, 1);
    }
    __threadfence();
  }
  __syncthreads();
}

// The timeout path of the grid barrier, run on purpose: one CTA arrives at a barrier whose count
// says that another arrival is still due (no other CTA exists), so the generation it waits on
// never advances; after `spins` polls it sets the timeout flag and leaves.
__global__ void kb_barrier_check(GridBar G, int spins) {
  if (threadIdx.x == 0) *G.count = 1;  // one phantom arrival: this CTA is never the last
  grid_barrier(G, spins);
  if (threadIdx.x == 0) *G.count = 0;
}

struct StageLists {
  const WorkItem* items[WL_COUNT];
  int n[WL_COUNT], total[WL_COUNT];
};

template <int ND, bool VISC, class R, bool SP>
__global__ void __launch_bounds__(kFusedBlock, sizeof(R) == 4 ? 896 / kFusedBlock : 384 / kFusedBlock)
    kb_stage(const BatchJob<R>* jobs, StageLists W, int stage, int fused_grad, GridBar G) {
  __shared__ BoundSlot<ND, R> slots[kFusedBlock];
  __shared__ int count;
  const int qin = stage == 3 ? 0 : stage;
  for_work(W.items[WL_PAD], W.n[WL_PAD], W.total[WL_PAD], [&](const WorkItem& it, int lb) {
    const BatchJob<R>& J = jobs[it.job];
    BATCH_CELL(J.pad);
    body_prim_halo<ND>(J.A, J.q[qin], J.dq[qin], i, j, k);
  });
  grid_barrier(G);
  if (!kFaceFormsG2<R> && fused_grad) {
    for_work(W.items[WL_GRAD1], W.n[WL_GRAD1], W.total[WL_GRAD1], [&](const WorkItem& it, int lb) {
      const BatchJob<R>& J = jobs[it.job];
      BATCH_CELL(J.grad1[it.sub]);
      body_grad12<ND>(J.A, it.sub, J.grad2[it.sub], i, j, k);
    });
  } else {
    for_work(W.items[WL_GRAD1], W.n[WL_GRAD1], W.total[WL_GRAD1], [&](const WorkItem& it, int lb) {
      const BatchJob<R>& J = jobs[it.job];
      BATCH_CELL(J.grad1[it.sub]);
      body_grad1<ND>(J.A, it.sub, i, j, k);
    });
    if constexpr (!kFaceFormsG2<R>) {
      grid_barrier(G);
      for_work(W.items[WL_GRAD2], W.n[WL_GRAD2], W.total[WL_GRAD2], [&](const WorkItem& it, int lb) {
        const BatchJob<R>& J = jobs[it.job];
        BATCH_CELL(J.grad2[it.sub]);
        body_grad2<ND>(J.A, it.sub, i, j, k);
      });
    }
  }
  grid_barrier(G);
  for_work(W.items[WL_FACE], W.n[WL_FACE], W.total[WL_FACE], [&](const WorkItem& it, int lb) {
    const BatchJob<R>& J = jobs[it.job];
    const long long t = (long long)lb * blockDim.x + threadIdx.x;
    const bool valid = t < box_size(J.faces[it.sub]);
    int i = 0, j = 0, k = 0;
    if (valid) box_coord(J.faces[it.sub], t, i, j, k);
    face_block<ND, VISC, false>(J.A, it.sub, valid, i, j, k, slots, &count);
  });
  grid_barrier(G);
  for_work(W.items[WL_INNER], W.n[WL_INNER], W.total[WL_INNER], [&](const WorkItem& it, int lb) {
    const BatchJob<R>& J = jobs[it.job];
    BATCH_CELL(J.inner);
    if (body_update<ND, false, R, SP>(J.U[stage], i, j, k)) atomicOr(J.err, 1);
  });
}

template <int ND, class R>
__global__ void __launch_bounds__(kBlock) kb_dt(const BatchJob<R>* jobs, const WorkItem* items, int n, int total) {
  // the minimum in the path's type and one conversion per block, as in k_dt
  __shared__ R wmin[kBlock / 32];
  phase_work(items, n, total, [&](const WorkItem& it, int lb) {
    const BatchJob<R>& J = jobs[it.job];
    const long long t = (long long)lb * blockDim.x + threadIdx.x;
    R v = R(HUGE_VAL);
    if (t < box_size(J.inner)) {
      int i, j, k;
      box_coord(J.inner, t, i, j, k);
      v = body_dt_r<ND, R>(J.D, i, j, k);
    }
    for (int off = 16; off > 0; off >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, off));
    __syncthreads();  // wmin of the previous block of this CTA has been read
    if ((threadIdx.x & 31) == 0) wmin[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
      R w = (threadIdx.x < blockDim.x / 32) ? wmin[threadIdx.x] : R(HUGE_VAL);
      for (int off = 16; off > 0; off >>= 1) w = fmin(w, __shfl_xor_sync(0xffffffffu, w, off));
      if (threadIdx.x == 0) atomicMin(J.dtbits, (unsigned long long)__double_as_longlong(fmin(1.0e300, double(w))));
    }
  });
}

// per member: 0 = reset the time-step minimum (CFL) or set the fixed step, 1 = dt from the minimum,
// 2 = advance the time
template <class R>
__global__ void kb_scalar(const BatchJob<R>* jobs, int n, int what) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n) return;
  const BatchJob<R>& J = jobs[m];
  if (what == 0) {
    if (J.cfl > 0.0) *J.dtbits = (unsigned long long)__double_as_longlong(1.0e300);
    else J.scal[S_DT] = -J.cfl;
  } else if (what == 1) {
    if (J.cfl > 0.0) J.scal[S_DT] = J.cfl * __longlong_as_double((long long)*J.dtbits);
  } else {
    J.scal[S_T] += J.scal[S_DT];
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
constexpr int kFaceBlockOptions[3] = {64, 128, 256};

struct KindKey {
  int nd, visc, prec, mov, ig4;
  bool operator==(const KindKey& o) const {
    return nd == o.nd && visc == o.visc && prec == o.prec && mov == o.mov && ig4 == o.ig4;
  }
};

struct Tuning {
  int face_block = 128;  // interfaces per tile
  int fused_grad = 0;    // 1: one fused gradient sweep
  int fused_stage = 0;   // 1: the whole right-hand side of a stage in one persistent cooperative launch
};

struct Kind {
  KindKey key;
  std::vector<gbr_ctx*> members;
  std::vector<double> cfl;
  size_t job_bytes = 0;
  char* d_jobs = nullptr;  // BatchJob<R>[members]
  WorkItem* d_items[WL_COUNT] = {};
  std::vector<WorkItem> items[WL_COUNT];
  int total[WL_COUNT] = {};
  // the interface items ordered by direction: direction d is items[WL_FACE][face_start[d] ..
  // face_start[d] + face_n[d]), blocks face_base[d] .. face_base[d] + face_total[d] of the list
  int face_start[3] = {}, face_n[3] = {}, face_base[3] = {}, face_total[3] = {};
  int face_dirs = 0;
  long long cells = 0;
  Tuning tune;
  unsigned* d_bar = nullptr;  // grid-barrier words of the fused stage kernel: count, generation, timeout
};

}  // namespace

struct gbr_batch {
  cudaStream_t stream;        // the members' stream: graphs and direct launches run here
  cudaStream_t cur = nullptr; // stream the enqueue functions issue to (the capture stream while capturing)
  cudaStream_t cap = nullptr; // private non-blocking stream the step graph is recorded on (the legacy
                              // default stream cannot be captured)
  std::vector<cudaStream_t> branch;  // one capture stream per kind: the kinds' steps are parallel
                                     // branches of the step graph
  char* ws;
  size_t ws_bytes;
  int max_members;
  std::vector<gbr_ctx*> members;
  std::vector<double> cfl;
  std::vector<Kind> kinds;
  bool dirty = true;
  int use_graph = 1;
  int autotune = 1;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  long long launches_per_step = 0;
  long long launches = 0;
  int sms = 0;
  std::vector<std::pair<long long, Tuning>> tune_cache;  // key: kind code * 64 + size class
  std::string last_error;
};

namespace {

gbr_status bfail(gbr_batch* b, gbr_status s, const std::string& m) {
  if (b) b->last_error = m;
  g_global_error = m;
  return s;
}

#define BK(expr, what)                                                                         \
  do {                                                                                         \
    cudaError_t _e = (expr);                                                                   \
    if (_e != cudaSuccess) return bfail(b, GBR_ECUDA, std::string(what) + ": " + cudaGetErrorString(_e)); \
  } while (0)

size_t batch_job_bytes() { return std::max(sizeof(BatchJob<double>), sizeof(BatchJob<float>)); }

size_t batch_ws_bytes(int max_members) {
  // per kind (at most 32: dimension, viscosity, precision, moving mesh, gradient scheme) the alignment
  // slack of its tables and its barrier words; per member one job record and at most
  // 1 + 3 + 3 + 3 + 1 + 1 + 1 items (pad, first derivatives cell by cell, second, interfaces,
  // inner, time step, first-derivative tiles: the capacities upload_kinds reserves)
  const size_t per_member = ((batch_job_bytes() + 255) & ~(size_t)255) + 13 * sizeof(WorkItem);
  return 32 * (size_t)(WL_COUNT + 2) * 256 + (size_t)max_members * (per_member + 256);
}

// a member's k_grad1v tiles (FP32 3D MEG6, aligned rows), balanced chunks of at most
// GBR_BATCH_G1V_CHUNK planes
#ifndef GBR_BATCH_G1V_CHUNK
#define GBR_BATCH_G1V_CHUNK 16
#endif
bool g1v_member(gbr_ctx* c, G1VPlan& P) {
  if (c->p.precision != GBR_PREC_MIXED || c->L.nd != 3 || c->p.gradient_scheme == GBR_GRAD_MIG4) return false;
  const RhsArgsT<float> A = rhs_args_r<float>(c, c->q[0]);
  const void* g1p[3] = {A.g1[0], A.g1[1], A.g1[2]};
  return g1v_plan(c->L, rhs_boxes(c->L), A.prim, A.temp, g1p, c->visc, -GBR_BATCH_G1V_CHUNK, P);
}

template <class R>
BatchJob<R> make_job(gbr_ctx* c, double cfl) {
  BatchJob<R> J;
  std::memset(&J, 0, sizeof J);
  const Layout& L = c->L;
  J.A = rhs_args_r<R>(c, c->q[0]);
  const double ca[3] = {1.0, 0.75, 1.0 / 3.0}, cb[3] = {0.0, 0.25, 2.0 / 3.0}, cc[3] = {1.0, 0.25, 2.0 / 3.0};
  for (int s = 0; s < 4; ++s) {
    UpdArgsT<R>& U = J.U[s];
    U.L = L;
    for (int d = 0; d < 3; ++d) U.flux[d] = static_cast<const R*>(c->flux[d]);
    U.jac = c->jac;
    U.jac32 = c->jac32;
    U.gcl = c->gcl;
    U.sigma = c->have_sponge ? c->sigma : nullptr;
    for (int v = 0; v < 5; ++v) U.qamb[v] = c->qamb[v];
    U.dt = c->scal + S_DT;
    if (s < 3) {
      // the same stage combinations as gbr_rk_step
      U.qs = c->q[s];
      U.q0 = c->q[0];
      U.out = (s == 2) ? c->q[0] : c->q[s + 1];
      U.ca = ca[s];
      U.cb = cb[s];
      U.cc = cc[s];
      U.mode = 1;
    } else {
      U.qs = c->q[0];
      U.q0 = c->q[0];
      U.out = c->q[1];
      U.ca = U.cb = 0.0;
      U.cc = 1.0;
      U.mode = 0;
    }
  }
  J.D = dt_args(c);  // the time metrics of a moving member (null for a static one)
  for (int s = 0; s < 3; ++s) J.q[s] = c->q[s];
  if (rk_in_increments(c)) {
    // the same increment form as gbr_rk_step: Q_s = Q^n + D_s, D1 and D2 in the stage buffers
    float* d1 = reinterpret_cast<float*>(c->q[1]);
    float* d2 = reinterpret_cast<float*>(c->q[2]);
    for (int s = 0; s < 3; ++s) {
      J.q[s] = c->q[0];
      J.U[s].qs = c->q[0];
    }
    J.dq[1] = d1;
    J.dq[2] = d2;
    J.U[0].dq_out = d1;
    J.U[0].out = nullptr;
    J.U[1].dq_in = d1;
    J.U[1].dq_out = d2;
    J.U[1].out = nullptr;
    J.U[2].dq_in = d2;
  }
  const RhsBoxes B = rhs_boxes(L);
  J.pad = pad_box(L, H, H);
  J.inner = B.inner;
  for (int d = 0; d < 3; ++d) {
    J.grad1[d] = B.grad1[d];
    J.grad2[d] = B.grad2[d];
    J.faces[d] = B.faces[d];
  }
  J.scal = c->scal;
  J.dtbits = reinterpret_cast<unsigned long long*>(c->scal + S_DTMIN);
  J.err = c->err;
  J.cfl = cfl;
  if constexpr (sizeof(R) == sizeof(float)) {
    G1VPlan P;
    if (g1v_member(c, P)) {
      J.g1u = P.U;
      J.g1v[0] = P.tiles_x;
      J.g1v[1] = P.tiles_y;
      J.g1v[2] = P.zchunk;
      J.g1v[3] = P.chunks;
    }
  }
  return J;
}

// xt > 0: the box's blocks under the transposed x-sweep mapping with WX = xt
void add_items(std::vector<WorkItem>& v, int& total, int job, int sub, const Box& box, int block, int xt = 0) {
  const int blocks = (int)(xt > 0 ? face_xt_blocks(box, block, xt) : (box_size(box) + block - 1) / block);
  if (blocks <= 0) return;
  v.push_back(WorkItem{job, sub, total, blocks});
  total += blocks;
}

void build_items(Kind& K) {
  for (int w = 0; w < WL_COUNT; ++w) {
    K.items[w].clear();
    K.total[w] = 0;
  }
  for (size_t m = 0; m < K.members.size(); ++m) {
    gbr_ctx* c = K.members[m];
    const Layout& L = c->L;
    const RhsBoxes B = rhs_boxes(L);
    const int jm = (int)m;
    // the fused stage kernel runs every phase with its one block size
    const int sb = K.tune.fused_stage ? kFusedBlock : kBlock;
    add_items(K.items[WL_PAD], K.total[WL_PAD], jm, 0, pad_box(L, H, H), sb);
    G1VPlan P;
    const bool tiles = !K.tune.fused_stage && g1v_member(c, P);
    if (tiles) {
      K.items[WL_G1V].push_back(WorkItem{jm, 0, K.total[WL_G1V], (int)P.blocks()});
      K.total[WL_G1V] += (int)P.blocks();
    }
    for (int d = 0; d < L.nd; ++d) {
      if (!tiles) add_items(K.items[WL_GRAD1], K.total[WL_GRAD1], jm, d, B.grad1[d], sb);
      add_items(K.items[WL_GRAD2], K.total[WL_GRAD2], jm, d, B.grad2[d], sb);
    }
    add_items(K.items[WL_INNER], K.total[WL_INNER], jm, 0, B.inner, sb);
    if (K.cfl[m] > 0.0) add_items(K.items[WL_DT], K.total[WL_DT], jm, 0, B.inner, kBlock);
  }
  // interfaces: every member's x-sweep, then the y- and z-sweeps (one launch per direction)
  const int fb = K.tune.fused_stage ? kFusedBlock : K.tune.face_block;
  // kb_face's 3D x-sweep mapping (the fused stage kernel keeps the linear one)
  const int xt = (K.tune.fused_stage || K.key.nd != 3) ? 0
                 : (K.key.prec == GBR_PREC_MIXED ? GBR_FACE_XT_WX_F32 : GBR_FACE_XT_WX);
  K.face_dirs = 0;
  for (int d = 0; d < 3; ++d) {
    K.face_start[d] = (int)K.items[WL_FACE].size();
    K.face_base[d] = K.total[WL_FACE];
    for (size_t m = 0; m < K.members.size(); ++m) {
      const Layout& L = K.members[m]->L;
      if (d < L.nd)
        add_items(K.items[WL_FACE], K.total[WL_FACE], (int)m, d, rhs_boxes(L).faces[d], fb, d == 0 ? xt : 0);
    }
    K.face_n[d] = (int)K.items[WL_FACE].size() - K.face_start[d];
    K.face_total[d] = K.total[WL_FACE] - K.face_base[d];
    if (K.face_n[d] > 0) ++K.face_dirs;
  }
}

// co-resident CTAs of a kernel, the grid of its persistent launch
template <class KernelT>
int resident_ctas(gbr_batch* b, KernelT kernel, int block) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, 0) != cudaSuccess || per_sm < 1) per_sm = 1;
  return per_sm * b->sms;
}

template <class KernelT>
unsigned persistent_grid(gbr_batch* b, KernelT kernel, int block, int total) {
  return (unsigned)std::max(1, std::min(total, resident_ctas(b, kernel, block)));
}

// the grid of a phase kernel (phase_work)
template <class KernelT>
unsigned phase_grid(gbr_batch* b, KernelT kernel, int block, int total) {
  return GBR_BATCH_ONE ? (unsigned)std::max(1, total) : persistent_grid(b, kernel, block, total);
}

// one launch per sweep direction, each over that direction's range of the interface items
template <int ND, bool VISC, bool MOV, class R, int BS>
gbr_status launch_face_kind(gbr_batch* b, const Kind& K, const BatchJob<R>* jobs, long long& launches) {
  auto one = [&](auto dd) -> gbr_status {
    constexpr int D = decltype(dd)::value;
    if (K.face_n[D] == 0) return GBR_OK;
    auto kern = kb_face<ND, VISC, MOV, R, BS, D>;
    const unsigned g = GBR_BATCH_FACE_ONE ? (unsigned)K.face_total[D] : persistent_grid(b, kern, BS, K.face_total[D]);
    kern<<<g, BS, 0, b->cur>>>(jobs, K.d_items[WL_FACE] + K.face_start[D], K.face_n[D], K.face_total[D],
                               K.face_base[D]);
    BK(cudaGetLastError(), "kb_face");
    ++launches;
    return GBR_OK;
  };
  gbr_status s = one(std::integral_constant<int, 0>{});
  if (s == GBR_OK) s = one(std::integral_constant<int, 1>{});
  if constexpr (ND == 3)
    if (s == GBR_OK) s = one(std::integral_constant<int, 2>{});
  return s;
}

// work of one member launched on the batch's current stream (its geometry, its IG4 solves),
// counted in `launches` through the member's own launch counter
template <class Fn>
gbr_status member_launches(gbr_batch* b, gbr_ctx* c, long long& launches, Fn fn) {
  const long long before = c->launches;
  const gbr_status s = fn();
  launches += c->launches - before;
  if (s != GBR_OK) return bfail(b, s, c->last_error);
  return GBR_OK;
}

// the geometry of every member with a prescribed motion at the stage time t^n + stage_c dt
gbr_status enqueue_geometry(gbr_batch* b, const Kind& K, double stage_c, long long& launches) {
  for (gbr_ctx* c : K.members) {
    if (!c->have_motion) continue;
    gbr_status s = member_launches(b, c, launches, [&] {
      gbr_status r = run_motion(c, stage_c, b->cur);
      return r == GBR_OK ? run_geometry(c, b->cur) : r;
    });
    if (s != GBR_OK) return s;
  }
  return GBR_OK;
}

// the fused stage kernel of a kind: one cooperative launch of as many CTAs as are resident
template <int ND, bool VISC, class R, bool SP>
gbr_status launch_stage_fused(gbr_batch* b, const Kind& K, const BatchJob<R>* jobs, int stage) {
  auto kern = kb_stage<ND, VISC, R, SP>;
  StageLists W;
  for (int w = 0; w < WL_COUNT; ++w) {
    W.items[w] = K.d_items[w];
    W.n[w] = (int)K.items[w].size();
    W.total[w] = K.total[w];
  }
  GridBar G{K.d_bar, K.d_bar + 1, reinterpret_cast<int*>(K.d_bar + 2)};
  int fg = K.tune.fused_grad;
  const int grid = resident_ctas(b, kern, kFusedBlock);
  void* args[] = {(void*)&jobs, (void*)&W, (void*)&stage, (void*)&fg, (void*)&G};
  BK(cudaLaunchCooperativeKernel((const void*)kern, dim3((unsigned)grid), dim3(kFusedBlock), args, 0, b->cur), "kb_stage");
  return GBR_OK;
}

// the right-hand side of `stage` (0..3, 3 = autotuning evaluation) for one kind
template <int ND, bool VISC, bool MOV, class R>
gbr_status enqueue_rhs(gbr_batch* b, const Kind& K, int stage, long long& launches) {
  const BatchJob<R>* jobs = reinterpret_cast<const BatchJob<R>*>(K.d_jobs);
  cudaStream_t st = b->cur;
  if constexpr (!MOV) {
    if (K.tune.fused_stage && !K.key.ig4) {
      bool sponge = false;
      for (gbr_ctx* m : K.members) sponge |= m->have_sponge;
      ++launches;
      return sponge ? launch_stage_fused<ND, VISC, R, true>(b, K, jobs, stage)
                    : launch_stage_fused<ND, VISC, R, false>(b, K, jobs, stage);
    }
  }
  const int qin = stage == 3 ? 0 : stage;
  {
    auto kern = kb_prim_halo<ND, R>;
    kern<<<phase_grid(b, kern, kBlock, K.total[WL_PAD]), kBlock, 0, st>>>(
        jobs, K.d_items[WL_PAD], (int)K.items[WL_PAD].size(), K.total[WL_PAD], qin);
    BK(cudaGetLastError(), "kb_prim_halo");
  }
  if (K.key.ig4) {
    // MIG4: each member's line solves (their tiles and launch shapes are per member), then, on the
    // FP64 path, the second derivatives of the whole kind in one launch
    for (gbr_ctx* c : K.members) {
      gbr_status s = member_launches(b, c, launches,
                                     [&] { return launch_ig4_grads<ND, R>(c, rhs_args_r<R>(c, c->q[0]), st); });
      if (s != GBR_OK) return s;
    }
    ++launches;
    if constexpr (!kFaceFormsG2<R>) {
      auto k2 = kb_grad2<ND, R>;
      k2<<<phase_grid(b, k2, kBlock, K.total[WL_GRAD2]), kBlock, 0, st>>>(
          jobs, K.d_items[WL_GRAD2], (int)K.items[WL_GRAD2].size(), K.total[WL_GRAD2]);
      BK(cudaGetLastError(), "kb_grad2");
      ++launches;
    }
  } else if constexpr (kFaceFormsG2<R>) {
    // FP32: the interface kernel forms f'' itself; first derivatives cell by cell and, for the
    // members on WL_G1V, by k_grad1v's tiles
    ++launches;  // the primitive pass above
    if (!K.items[WL_GRAD1].empty()) {
      auto k1 = kb_grad1<ND, R>;
      k1<<<phase_grid(b, k1, kBlock, K.total[WL_GRAD1]), kBlock, 0, st>>>(
          jobs, K.d_items[WL_GRAD1], (int)K.items[WL_GRAD1].size(), K.total[WL_GRAD1]);
      BK(cudaGetLastError(), "kb_grad1");
      ++launches;
    }
    if constexpr (ND == 3 && sizeof(R) == sizeof(float)) {
      if (!K.items[WL_G1V].empty()) {
        auto kv = kb_grad1v;
        kv<<<phase_grid(b, kv, kGVX * kGVY, K.total[WL_G1V]), kGVX * kGVY, 0, st>>>(
            jobs, K.d_items[WL_G1V], (int)K.items[WL_G1V].size(), K.total[WL_G1V]);
        BK(cudaGetLastError(), "kb_grad1v");
        ++launches;
      }
    }
  } else if (K.tune.fused_grad) {
    auto kern = kb_grad12<ND, R>;
    kern<<<phase_grid(b, kern, kBlock, K.total[WL_GRAD1]), kBlock, 0, st>>>(
        jobs, K.d_items[WL_GRAD1], (int)K.items[WL_GRAD1].size(), K.total[WL_GRAD1]);
    BK(cudaGetLastError(), "kb_grad12");
    launches += 2;
  } else {
    auto k1 = kb_grad1<ND, R>;
    k1<<<phase_grid(b, k1, kBlock, K.total[WL_GRAD1]), kBlock, 0, st>>>(
        jobs, K.d_items[WL_GRAD1], (int)K.items[WL_GRAD1].size(), K.total[WL_GRAD1]);
    BK(cudaGetLastError(), "kb_grad1");
    auto k2 = kb_grad2<ND, R>;
    k2<<<phase_grid(b, k2, kBlock, K.total[WL_GRAD2]), kBlock, 0, st>>>(
        jobs, K.d_items[WL_GRAD2], (int)K.items[WL_GRAD2].size(), K.total[WL_GRAD2]);
    BK(cudaGetLastError(), "kb_grad2");
    launches += 3;
  }
  gbr_status s;
  switch (K.tune.face_block) {
    case 64: s = launch_face_kind<ND, VISC, MOV, R, 64>(b, K, jobs, launches); break;
    case 256: s = launch_face_kind<ND, VISC, MOV, R, 256>(b, K, jobs, launches); break;
    default: s = launch_face_kind<ND, VISC, MOV, R, 128>(b, K, jobs, launches); break;
  }
  if (s != GBR_OK) return s;
  {
    // the sponge-capable instantiation only when a member of the kind has a sponge
    bool sponge = false;
    for (gbr_ctx* m : K.members) sponge |= m->have_sponge;
    auto kern = sponge ? kb_update<ND, MOV, R, true> : kb_update<ND, MOV, R, false>;
    kern<<<phase_grid(b, kern, kBlock, K.total[WL_INNER]), kBlock, 0, st>>>(
        jobs, K.d_items[WL_INNER], (int)K.items[WL_INNER].size(), K.total[WL_INNER], stage);
    BK(cudaGetLastError(), "kb_update");
  }
  launches += 1;  // the update (launch_face_kind counted the interface launches)
  return GBR_OK;
}

template <int ND, bool VISC, bool MOV, class R>
gbr_status enqueue_step_kind(gbr_batch* b, const Kind& K, long long& launches) {
  const BatchJob<R>* jobs = reinterpret_cast<const BatchJob<R>*>(K.d_jobs);
  cudaStream_t st = b->cur;
  const int n = (int)K.members.size();
  const unsigned gs = (unsigned)((n + 127) / 128);
  gbr_status sg;
  // as gbr_rk_step: the geometry at t^n (moving members), then the time step from Q^n
  if (MOV && (sg = enqueue_geometry(b, K, 0.0, launches)) != GBR_OK) return sg;
  kb_scalar<R><<<gs, 128, 0, st>>>(jobs, n, 0);
  BK(cudaGetLastError(), "kb_scalar");
  launches += 2;
  if (K.total[WL_DT] > 0) {
    auto kern = kb_dt<ND, R>;
    kern<<<phase_grid(b, kern, kBlock, K.total[WL_DT]), kBlock, 0, st>>>(
        jobs, K.d_items[WL_DT], (int)K.items[WL_DT].size(), K.total[WL_DT]);
    BK(cudaGetLastError(), "kb_dt");
    ++launches;
  }
  kb_scalar<R><<<gs, 128, 0, st>>>(jobs, n, 1);
  BK(cudaGetLastError(), "kb_scalar");
  const double stage_c[3] = {0.0, 1.0, 0.5};  // stage times t^n + c dt of SSP-RK3
  for (int stage = 0; stage < 3; ++stage) {
    if (MOV && stage > 0 && (sg = enqueue_geometry(b, K, stage_c[stage], launches)) != GBR_OK) return sg;
    gbr_status s = enqueue_rhs<ND, VISC, MOV, R>(b, K, stage, launches);
    if (s != GBR_OK) return s;
  }
  kb_scalar<R><<<gs, 128, 0, st>>>(jobs, n, 2);
  BK(cudaGetLastError(), "kb_scalar");
  ++launches;
  return GBR_OK;
}

// dispatch on the kind's template parameters
template <int ND, bool VISC, class Fn>
gbr_status dispatch_mov(const KindKey& k, Fn& fn) {
  if (k.mov) return k.prec ? fn.template run<ND, VISC, true, float>() : fn.template run<ND, VISC, true, double>();
  return k.prec ? fn.template run<ND, VISC, false, float>() : fn.template run<ND, VISC, false, double>();
}

template <class Fn>
gbr_status dispatch_kind(const KindKey& k, Fn fn) {
  if (k.nd == 3) return k.visc ? dispatch_mov<3, true>(k, fn) : dispatch_mov<3, false>(k, fn);
  return k.visc ? dispatch_mov<2, true>(k, fn) : dispatch_mov<2, false>(k, fn);
}

struct StepFn {
  gbr_batch* b;
  const Kind* K;
  long long* launches;
  template <int ND, bool VISC, bool MOV, class R>
  gbr_status run() { return enqueue_step_kind<ND, VISC, MOV, R>(b, *K, *launches); }
};

struct RhsFn {
  gbr_batch* b;
  const Kind* K;
  long long* launches;
  template <int ND, bool VISC, bool MOV, class R>
  gbr_status run() { return enqueue_rhs<ND, VISC, MOV, R>(b, *K, 3, *launches); }
};

struct UploadFn {
  gbr_batch* b;
  Kind* K;
  std::vector<char>* host;
  template <int ND, bool VISC, bool MOV, class R>
  gbr_status run() {
    const size_t n = K->members.size();
    host->assign(n * sizeof(BatchJob<R>), 0);
    for (size_t m = 0; m < n; ++m) {
      BatchJob<R> J = make_job<R>(K->members[m], K->cfl[m]);
      std::memcpy(host->data() + m * sizeof(BatchJob<R>), &J, sizeof J);
    }
    K->job_bytes = host->size();
    return GBR_OK;
  }
};

int kind_code(const KindKey& k) { return (k.nd - 2) * 16 + k.visc * 8 + k.prec * 4 + k.mov * 2 + k.ig4; }

int size_class(long long cells) {
  int c = 0;
  while (cells > 1) {
    cells >>= 1;
    ++c;
  }
  return c;
}

// lay out the kinds' tables in the batch workspace and copy them to the device
gbr_status upload_kinds(gbr_batch* b) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    off = (off + 255) & ~(size_t)255;
    char* p = b->ws + off;
    off += bytes;
    return p;
  };
  std::vector<char> host;
  for (Kind& K : b->kinds) {
    build_items(K);
    UploadFn up{b, &K, &host};
    gbr_status s = dispatch_kind(K.key, up);
    if (s != GBR_OK) return s;
    K.d_jobs = take(K.job_bytes);
    K.d_bar = reinterpret_cast<unsigned*>(take(4 * sizeof(unsigned)));
    if (off > b->ws_bytes) return bfail(b, GBR_ENOMEM, "batch workspace too small");
    BK(cudaMemsetAsync(K.d_bar, 0, 4 * sizeof(unsigned), b->stream), "barrier words");
    BK(cudaMemcpyAsync(K.d_jobs, host.data(), K.job_bytes, cudaMemcpyHostToDevice, b->stream), "upload jobs");
    for (int w = 0; w < WL_COUNT; ++w) {
      // the autotuner's candidates reuse these buffers: a member's first derivatives are one
      // WL_G1V item or nd WL_GRAD1 items, depending on the candidate
      size_t cap = K.items[w].size();
      if (w == WL_GRAD1) cap = std::max(cap, K.members.size() * (size_t)K.key.nd);
      if (w == WL_G1V) cap = std::max(cap, K.members.size());
      const size_t bytes = std::max<size_t>(1, cap) * sizeof(WorkItem);
      K.d_items[w] = reinterpret_cast<WorkItem*>(take(bytes));
      if (off > b->ws_bytes) return bfail(b, GBR_ENOMEM, "batch workspace too small");
      if (!K.items[w].empty())
        BK(cudaMemcpyAsync(K.d_items[w], K.items[w].data(), K.items[w].size() * sizeof(WorkItem),
                           cudaMemcpyHostToDevice, b->stream),
           "upload work list");
    }
    // the host vectors are reused: finish the copies before the next kind overwrites them
    BK(cudaStreamSynchronize(b->stream), "upload sync");
  }
  return GBR_OK;
}

gbr_status enqueue_step(gbr_batch* b, long long& launches) {
  for (const Kind& K : b->kinds) {
    StepFn fn{b, &K, &launches};
    gbr_status s = dispatch_kind(K.key, fn);
    if (s != GBR_OK) return s;
  }
  return GBR_OK;
}

// time the stage-1 right-hand side of one kind under each tuning; keep the fastest
gbr_status autotune_kind(gbr_batch* b, Kind& K) {
  const long long key = (long long)kind_code(K.key) * 64 + size_class(K.cells);
  for (auto& e : b->tune_cache)
    if (e.first == key) {
      K.tune = e.second;
      return GBR_OK;
    }
  cudaEvent_t e0, e1;
  BK(cudaEventCreate(&e0), "event");
  BK(cudaEventCreate(&e1), "event");
  Tuning best;
  float best_ms = 1e30f;
  std::vector<char> host;
  // candidates: the phase kernels with each interface tile size, and (static MEG6 kinds) the
  // fused stage kernel; the gradient sweep is a choice of the FP64 path only (FP32 forms f'' in the
  // interface kernel; MIG4 kinds solve their first derivatives per member)
  const bool can_fuse = !K.key.mov && !K.key.ig4;
  for (int cand = 0; cand < 4; ++cand) {
    const int fb = cand < 3 ? kFaceBlockOptions[cand] : kFusedBlock;
    const int stage_fused = cand == 3 ? 1 : 0;
    if (stage_fused && !can_fuse) continue;
    for (int fused = 0; fused < ((K.key.prec == GBR_PREC_MIXED || K.key.ig4) ? 1 : 2); ++fused) {
      K.tune.face_block = fb;
      K.tune.fused_grad = fused;
      K.tune.fused_stage = stage_fused;
      build_items(K);
      // the work lists of this candidate (their lengths do not depend on the block sizes)
      for (int w = 0; w < WL_COUNT; ++w)
        if (!K.items[w].empty())
          BK(cudaMemcpyAsync(K.d_items[w], K.items[w].data(), K.items[w].size() * sizeof(WorkItem),
                             cudaMemcpyHostToDevice, b->stream),
             "upload work list");
      long long dummy = 0;
      RhsFn fn{b, &K, &dummy};
      b->cur = b->stream;
      gbr_status s = dispatch_kind(K.key, fn);  // warm-up
      if (s != GBR_OK) return s;
      BK(cudaEventRecord(e0, b->stream), "event");
      for (int r = 0; r < 3; ++r)
        if ((s = dispatch_kind(K.key, fn)) != GBR_OK) return s;
      BK(cudaEventRecord(e1, b->stream), "event");
      BK(cudaEventSynchronize(e1), "event sync");
      float ms = 0.f;
      BK(cudaEventElapsedTime(&ms, e0, e1), "event time");
      if (ms < best_ms) {
        best_ms = ms;
        best = K.tune;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  K.tune = best;
  b->tune_cache.push_back({key, best});
  return GBR_OK;
}

gbr_status rebuild(gbr_batch* b) {
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  if (b->graph) {
    cudaGraphDestroy(b->graph);
    b->graph = nullptr;
  }
  b->kinds.clear();
  for (size_t m = 0; m < b->members.size(); ++m) {
    gbr_ctx* c = b->members[m];
    KindKey key{c->L.nd, c->visc ? 1 : 0, c->p.precision == GBR_PREC_MIXED ? 1 : 0, c->mov ? 1 : 0,
                c->p.gradient_scheme == GBR_GRAD_MIG4 ? 1 : 0};
    Kind* K = nullptr;
    for (Kind& x : b->kinds)
      if (x.key == key) K = &x;
    if (!K) {
      b->kinds.push_back(Kind());
      K = &b->kinds.back();
      K->key = key;
    }
    K->members.push_back(c);
    K->cfl.push_back(b->cfl[m]);
    K->cells += c->L.ncells;
  }
  for (Kind& K : b->kinds) {
    const long long key = (long long)kind_code(K.key) * 64 + size_class(K.cells);
    for (auto& e : b->tune_cache)
      if (e.first == key) K.tune = e.second;
  }
  if (b->autotune == 2)  // the fused stage kernel wherever it applies, untimed
    for (Kind& K : b->kinds)
      if (!K.key.mov && !K.key.ig4) {
        K.tune.fused_stage = 1;
        K.tune.face_block = kFusedBlock;
        K.tune.fused_grad = 0;
      }
  gbr_status s = upload_kinds(b);
  if (s != GBR_OK) return s;
  if (b->autotune == 1) {
    for (Kind& K : b->kinds)
      if ((s = autotune_kind(b, K)) != GBR_OK) return s;
    if ((s = upload_kinds(b)) != GBR_OK) return s;
  }
  long long launches = 0;
  if (b->use_graph && !b->members.empty()) {
    if (!b->cap) BK(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking), "capture stream");
    b->cur = b->cap;
    BK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
    if (b->kinds.size() > 1) {
      // the kinds share no data: each kind's step is a branch forked from and joined to the capture
      // stream, so a kind whose launches do not fill the GPU overlaps the others
      while (b->branch.size() < b->kinds.size()) {
        cudaStream_t x = nullptr;
        BK(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking), "branch stream");
        b->branch.push_back(x);
      }
      std::vector<cudaEvent_t> ev(b->kinds.size() + 1, nullptr);
      for (auto& x : ev) BK(cudaEventCreateWithFlags(&x, cudaEventDisableTiming), "branch event");
      BK(cudaEventRecord(ev[0], b->cap), "fork");
      for (size_t k = 0; k < b->kinds.size() && s == GBR_OK; ++k) {
        BK(cudaStreamWaitEvent(b->branch[k], ev[0], 0), "fork wait");
        b->cur = b->branch[k];
        StepFn fn{b, &b->kinds[k], &launches};
        s = dispatch_kind(b->kinds[k].key, fn);
        BK(cudaEventRecord(ev[k + 1], b->branch[k]), "join");
        BK(cudaStreamWaitEvent(b->cap, ev[k + 1], 0), "join wait");
      }
      b->cur = b->cap;
      cudaGraph_t g0 = nullptr;
      cudaError_t e0 = cudaStreamEndCapture(b->cap, &g0);
      for (auto& x : ev) cudaEventDestroy(x);
      b->cur = b->stream;
      if (s != GBR_OK || e0 != cudaSuccess) {
        if (g0) cudaGraphDestroy(g0);
        if (s != GBR_OK) return s;
        BK(e0, "end capture");
      }
      b->graph = g0;
      BK(cudaGraphInstantiate(&b->exec, b->graph, 0), "graph instantiate");
      b->launches_per_step = launches;
      b->dirty = false;
      return GBR_OK;
    }
    s = enqueue_step(b, launches);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->cap, &g);
    b->cur = b->stream;
    if (s != GBR_OK) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    BK(e, "end capture");
    b->graph = g;
    BK(cudaGraphInstantiate(&b->exec, b->graph, 0), "graph instantiate");
  } else {
    // count the launches of one step without running it; a kind with per-member work (moving
    // meshes, MIG4) is counted when its first step is enqueued (gbr_batch_step)
    for (const Kind& K : b->kinds) {
      if (K.key.mov || K.key.ig4) {
        launches = -1;
        break;
      }
      // phase kernels: primitives, gradients (one or two), one interface launch per direction, update
      const int grads = K.key.prec == GBR_PREC_MIXED
                            ? (K.items[WL_GRAD1].empty() ? 0 : 1) + (K.items[WL_G1V].empty() ? 0 : 1)
                            : (K.tune.fused_grad ? 1 : 2);
      const int per_stage = K.tune.fused_stage ? 1 : 2 + grads + K.face_dirs;
      launches += 3 + (K.total[WL_DT] > 0 ? 1 : 0) + 3 * per_stage;
    }
  }
  b->launches_per_step = launches;
  b->dirty = false;
  return GBR_OK;
}

}  // namespace

extern "C" {

size_t gbr_batch_workspace_bytes(int max_members) {
  if (max_members < 1) return 0;
  return batch_ws_bytes(max_members);
}

gbr_status gbr_batch_create(int max_members, void* d_workspace, size_t ws_bytes, void* stream, gbr_batch** out) {
  if (!out) return bfail(nullptr, GBR_EINVAL, "null output pointer");
  *out = nullptr;
  if (max_members < 1) return bfail(nullptr, GBR_EINVAL, "max_members must be positive");
  if (!d_workspace || ((uintptr_t)d_workspace & 255)) return bfail(nullptr, GBR_EINVAL, "workspace must be 256-byte aligned");
  if (ws_bytes < batch_ws_bytes(max_members)) return bfail(nullptr, GBR_ENOMEM, "batch workspace too small");
  gbr_batch* b = new gbr_batch();
  b->stream = (cudaStream_t)stream;
  b->cur = b->stream;
  b->ws = (char*)d_workspace;
  b->ws_bytes = ws_bytes;
  b->max_members = max_members;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || b->sms < 1) {
    delete b;
    return bfail(nullptr, GBR_ECUDA, "device query failed");
  }
  *out = b;
  return GBR_OK;
}

gbr_status gbr_batch_set_options(gbr_batch* b, int use_graph, int autotune) {
  if (!b) return bfail(b, GBR_EINVAL, "null batch");
  if (autotune < 0 || autotune > 2) return bfail(b, GBR_EINVAL, "autotune must be 0, 1 or 2");
  b->use_graph = use_graph ? 1 : 0;
  b->autotune = autotune;
  b->dirty = true;
  return GBR_OK;
}

gbr_status gbr_batch_add(gbr_batch* b, gbr_ctx* c, double cfl_or_neg_dt) {
  if (!b || !c) return bfail(b, GBR_EINVAL, "null argument");
  if (!(cfl_or_neg_dt != 0.0) || std::isnan(cfl_or_neg_dt)) return bfail(b, GBR_EINVAL, "cfl_or_neg_dt must be nonzero");
  if ((int)b->members.size() >= b->max_members) return bfail(b, GBR_ENOMEM, "batch is full");
  if (!c->metrics_ready) return bfail(b, GBR_ESTATE, "metrics not computed");
  if (c->stream != b->stream) return bfail(b, GBR_EINVAL, "the context must use the batch's stream");
  for (gbr_ctx* x : b->members)
    if (x == c) return bfail(b, GBR_EINVAL, "context already in the batch");
  b->members.push_back(c);
  b->cfl.push_back(cfl_or_neg_dt);
  b->dirty = true;
  return GBR_OK;
}

gbr_status gbr_batch_remove(gbr_batch* b, gbr_ctx* c) {
  if (!b || !c) return bfail(b, GBR_EINVAL, "null argument");
  for (size_t m = 0; m < b->members.size(); ++m)
    if (b->members[m] == c) {
      b->members.erase(b->members.begin() + m);
      b->cfl.erase(b->cfl.begin() + m);
      b->dirty = true;
      return GBR_OK;
    }
  return bfail(b, GBR_EINVAL, "context is not in the batch");
}

gbr_status gbr_batch_step(gbr_batch* b, int n_steps) {
  if (!b) return bfail(b, GBR_EINVAL, "null batch");
  if (n_steps < 0) return bfail(b, GBR_EINVAL, "n_steps must be non-negative");
  if (b->members.empty() || n_steps == 0) return GBR_OK;
  gbr_status s;
  if (b->dirty && (s = rebuild(b)) != GBR_OK) return s;
  for (int r = 0; r < n_steps; ++r) {
    if (b->exec) {
      BK(cudaGraphLaunch(b->exec, b->stream), "graph launch");
      b->launches += b->launches_per_step;
    } else {
      long long count = 0;
      b->cur = b->stream;
      if ((s = enqueue_step(b, count)) != GBR_OK) return s;
      b->launches_per_step = count;
      b->launches += count;
    }
  }
  return GBR_OK;
}

gbr_status gbr_batch_sync(gbr_batch* b, double timeout_s, int* bad_member) {
  if (!b) return bfail(b, GBR_EINVAL, "null batch");
  if (bad_member) *bad_member = -1;
  auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cudaError_t e = cudaStreamQuery(b->stream);
    if (e == cudaSuccess) break;
    if (e != cudaErrorNotReady) return bfail(b, GBR_ECUDA, std::string("stream query: ") + cudaGetErrorString(e));
    const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (timeout_s > 0.0 && el > timeout_s) return bfail(b, GBR_ETIMEOUT, "stream did not drain before the deadline");
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  for (const Kind& K : b->kinds) {
    if (!K.d_bar) continue;
    int tmo = 0;
    BK(cudaMemcpy(&tmo, K.d_bar + 2, sizeof(int), cudaMemcpyDeviceToHost), "read timeout flag");
    if (tmo) return bfail(b, GBR_ETIMEOUT, "a grid barrier of the fused stage kernel did not complete in time");
  }
  for (size_t m = 0; m < b->members.size(); ++m) {
    int err = 0;
    BK(cudaMemcpy(&err, b->members[m]->err, sizeof(int), cudaMemcpyDeviceToHost), "read error flag");
    if (err) {
      if (bad_member) *bad_member = (int)m;
      return bfail(b, GBR_ENONFINITE, "member " + std::to_string(m) + ": non-finite state or non-positive density");
    }
  }
  return GBR_OK;
}

gbr_status gbr_batch_info(gbr_batch* b, int* members, int* kinds, long long* launches_per_step, long long* launches) {
  if (!b) return bfail(b, GBR_EINVAL, "null batch");
  if (b->dirty && !b->members.empty()) {
    gbr_status s = rebuild(b);
    if (s != GBR_OK) return s;
  }
  if (members) *members = (int)b->members.size();
  if (kinds) *kinds = (int)b->kinds.size();
  if (launches_per_step) *launches_per_step = b->launches_per_step;
  if (launches) *launches = b->launches;
  return GBR_OK;
}

gbr_status gbr_batch_tuning(gbr_batch* b, int kind, int* nd, int* viscous, int* precision, int* face_block,
                            int* fused_grad, int* fused_stage) {
  if (!b) return bfail(b, GBR_EINVAL, "null batch");
  if (kind < 0 || kind >= (int)b->kinds.size()) return bfail(b, GBR_EINVAL, "no such kind");
  const Kind& K = b->kinds[kind];
  if (nd) *nd = K.key.nd;
  if (viscous) *viscous = K.key.visc;
  if (precision) *precision = K.key.prec;
  if (face_block) *face_block = K.tune.face_block;
  if (fused_grad) *fused_grad = K.tune.fused_grad;
  if (fused_stage) *fused_stage = K.tune.fused_stage;
  return GBR_OK;
}

gbr_status gbr_batch_check_barrier(gbr_batch* b, int polls) {
  if (!b) return bfail(b, GBR_EINVAL, "null batch");
  if (polls < 1 || polls > kGridBarSpin) return bfail(b, GBR_EINVAL, "polls out of range");
  if (b->dirty && !b->members.empty()) {
    gbr_status s = rebuild(b);
    if (s != GBR_OK) return s;
  }
  if (b->kinds.empty() || !b->kinds[0].d_bar) return bfail(b, GBR_ESTATE, "the batch has no members");
  unsigned* w = b->kinds[0].d_bar;
  kb_barrier_check<<<1, 32, 0, b->stream>>>(GridBar{w, w + 1, reinterpret_cast<int*>(w + 2)}, polls);
  BK(cudaGetLastError(), "kb_barrier_check");
  return GBR_OK;
}

const char* gbr_batch_last_error(const gbr_batch* b) { return b ? b->last_error.c_str() : g_global_error.c_str(); }

void gbr_batch_destroy(gbr_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (cudaStream_t x : b->branch) cudaStreamDestroy(x);
  delete b;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Device-memory arena: host bookkeeping of a caller-owned device range, used to
// admit jobs by their HBM footprint (gbr_workspace_bytes).  First fit over the
// free holes in address order, 256-byte granules, neighbours merged on free.
// Nothing here touches the device.
// ---------------------------------------------------------------------------
#include <map>

struct gbr_arena {
  uintptr_t base;
  size_t bytes;
  std::map<size_t, size_t> free_;  // offset -> length
  std::map<size_t, size_t> used_;  // offset -> length
  std::string last_error;
};

extern "C" {

gbr_status gbr_arena_create(void* d_base, size_t bytes, gbr_arena** out) {
  if (!out) return bfail(nullptr, GBR_EINVAL, "null output pointer");
  *out = nullptr;
  if (!d_base || ((uintptr_t)d_base & 255)) return bfail(nullptr, GBR_EINVAL, "arena base must be 256-byte aligned");
  bytes &= ~(size_t)255;
  if (bytes == 0) return bfail(nullptr, GBR_EINVAL, "empty arena");
  gbr_arena* a = new gbr_arena();
  a->base = (uintptr_t)d_base;
  a->bytes = bytes;
  a->free_[0] = bytes;
  *out = a;
  return GBR_OK;
}

gbr_status gbr_arena_alloc(gbr_arena* a, size_t bytes, void** ptr) {
  if (!a || !ptr) return bfail(nullptr, GBR_EINVAL, "null argument");
  *ptr = nullptr;
  if (bytes == 0) return bfail(nullptr, GBR_EINVAL, "zero-byte allocation");
  const size_t need = (bytes + 255) & ~(size_t)255;
  for (auto it = a->free_.begin(); it != a->free_.end(); ++it) {
    if (it->second < need) continue;
    const size_t off = it->first, len = it->second;
    a->free_.erase(it);
    if (len > need) a->free_[off + need] = len - need;
    a->used_[off] = need;
    *ptr = (void*)(a->base + off);
    return GBR_OK;
  }
  a->last_error = "no free range of " + std::to_string(need) + " bytes";
  return GBR_ENOMEM;
}

gbr_status gbr_arena_free(gbr_arena* a, void* ptr) {
  if (!a || !ptr) return bfail(nullptr, GBR_EINVAL, "null argument");
  const uintptr_t p = (uintptr_t)ptr;
  if (p < a->base || p >= a->base + a->bytes) return bfail(nullptr, GBR_EINVAL, "pointer outside the arena");
  const size_t off = p - a->base;
  auto u = a->used_.find(off);
  if (u == a->used_.end()) return bfail(nullptr, GBR_EINVAL, "pointer not allocated from this arena");
  size_t start = off, len = u->second;
  a->used_.erase(u);
  auto next = a->free_.lower_bound(start);
  if (next != a->free_.end() && next->first == start + len) {
    len += next->second;
    next = a->free_.erase(next);
  }
  if (next != a->free_.begin()) {
    auto prev = std::prev(next);
    if (prev->first + prev->second == start) {
      start = prev->first;
      len += prev->second;
      a->free_.erase(prev);
    }
  }
  a->free_[start] = len;
  return GBR_OK;
}

gbr_status gbr_arena_stats(const gbr_arena* a, size_t* used, size_t* free_total, size_t* largest_free, int* blocks) {
  if (!a) return bfail(nullptr, GBR_EINVAL, "null arena");
  size_t u = 0, f = 0, big = 0;
  for (auto& e : a->used_) u += e.second;
  for (auto& e : a->free_) {
    f += e.second;
    big = std::max(big, e.second);
  }
  if (used) *used = u;
  if (free_total) *free_total = f;
  if (largest_free) *largest_free = big;
  if (blocks) *blocks = (int)a->used_.size();
  return GBR_OK;
}

void gbr_arena_destroy(gbr_arena* a) { delete a; }

}  // extern "C"
