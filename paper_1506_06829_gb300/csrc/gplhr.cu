// libgplhr: host driver and C ABI of the GPLHR eigensolver (arXiv 1506.06829,
// Algorithm 2) on one GPU.  Device kernels are in kernels.cuh; the small dense
// QZ / Q-free factor algebra runs on the host (qz.cpp).
//
// Storage (Sec. 3.6: Z, U, AZ, BZ of n x s, s = (m+3)k): four n x s_max row-major
// complex blocks with s_max = (m0+3)k.  Column layout of Z (and of AZ, BZ):
//   [ V (k) | W (kk) | S_1 (kk) ... S_m (kk) | P (kk) ],  kk = k - q (soft locking),
// and U = [ Q (k) | Qhat (s - k) ].  For B = I, BZ is Z itself.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <climits>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <condition_variable>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/gplhr.h"
#include "kernels.cuh"
#include "persist.cuh"
#include "qz.h"
#include "qz_device.cuh"
#include "tc.cuh"

using gplhr::cd;
using gplhr::SqMat;

namespace {

// Message of the last failed context-free call (gplhr_create, gplhr_gram_noalloc, ...),
// per host thread: batched creation runs gplhr_create on several threads at once.
thread_local std::string g_create_error;

struct DevCsr {
  int* rowptr = nullptr;
  int* col = nullptr;
  void* val = nullptr;
  void* val32 = nullptr;  // FP32 copy of the values (mixed-precision mode)
  int dtype = GPLHR_R64;
  int64_t nnz = 0;
};

struct Blk {  // row-major block view
  double2* p;
  int ld;
};


}  // namespace

// Launches and copies of one device segment of an iteration, recorded instead of issued:
// the persistent batched iteration (gplhr_iterate_persistent) runs the segments of all
// its contexts in one kernel (persist.cuh).  Each op keeps the kernel kind, the grid the
// launch would have had (256 threads per CTA), its dynamic shared memory and its
// arguments (a byte range of args).  Host-to-device copies read staging the host filled
// before the segment, so they run before the kernel; device-to-host copies after it.
struct PkRecorder {
  struct Op {
    int kind, gx, gy;
    size_t smem, off, size;
  };
  struct Copy {
    void* dst;
    const void* src;
    size_t bytes;
  };
  std::vector<Op> ops;
  std::vector<unsigned char> args;
  std::vector<Copy> pre, post;
  void clear() {
    ops.clear();
    args.clear();
    pre.clear();
    post.clear();
  }
};

struct gplhr_ctx {
  // problem
  int n = 0, k = 0, m0 = 0, s_max = 0;
  cd sigma;
  bool hasB = false;
  DevCsr A, B, Tcsr;
  double normA = 1.0, normB = 1.0;
  int prec = GPLHR_PREC_NONE, bs = 1;
  double2* prec_data = nullptr;  // Jacobi diagonal or block-Jacobi inverse blocks
  float2* prec32 = nullptr;      // FP32 copy of the block-Jacobi inverse blocks (mixed mode)
  float2* X32 = nullptr;         // complex64 copy of a sparse product's input block (mixed mode)
  // options
  double tol = 1e-8;
  int maxit = 500;
  bool lock = true;
  bool recompute = false;  // AV, BV, AP, BP by sparse products instead of combinations
  bool mixed = false;      // mixed-precision mode requested
  bool bulk32 = false;     // currently in the FP32 bulk phase
  int fp32_iters = 0;      // iterations run in the bulk phase
  double best_res = 1e300; // stall detection for the bulk phase
  int since_best = 0;
  double switch_tol = 1e-5;
  int stall_iters = 5;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int num_sms = 152;
  // device buffers
  double2 *Z = nullptr, *AZ = nullptr, *BZ = nullptr, *U = nullptr;
  double2 *Pb = nullptr, *APb = nullptr, *BPb = nullptr;
  double2 *Rw = nullptr, *Tw1 = nullptr, *Tw2 = nullptr, *Tw3 = nullptr;  // Rw holds the residual
  double2 *dC1 = nullptr, *dC2 = nullptr, *dMBa = nullptr, *dMAa = nullptr;
  double2 *dYR = nullptr, *dYL = nullptr, *dPhiPsi = nullptr, *dGram = nullptr, *dProjC = nullptr;
  double2* dRinv = nullptr;  // 3 x s_max^2
  double2* dTrackC = nullptr;  // 3 x s_max^2: projection coefficients of each orth pass
  double2* dTrackR = nullptr;  // 3 x s_max^2: Cholesky factors of each orth pass
  double2* h_track = nullptr;  // pinned copies of the two above
  int* h_status = nullptr;
  size_t trk = 0;              // stride of the passes in dTrackC (>= s_max^2)
  bool factored = true;        // projected pencil from U's factors (one Gram)
  // deflation basis (gplhr_set_deflation): k1 right / left Schur vectors already computed;
  // the iteration then runs on ((I - Q1 Q1^*) A (I - V1 V1^*), (I - Q1 Q1^*) B (I - V1 V1^*))
  double2* dV1 = nullptr;
  double2* dQ1 = nullptr;
  int k1 = 0;
  // GPLHR-EIG (Algorithm 3): eigenvector iterate X (unit columns), A X, B X, and the
  // Rayleigh-quotient factors alpha_j = x_j^* A x_j, beta_j = x_j^* B x_j
  bool eig = false;
  double2 *eX = nullptr, *eAX = nullptr, *eBX = nullptr;
  std::vector<cd> ea, eb;
  int p_mode = 0;              // search directions P: 0 thick restart (Eq. P1), 1 LOBPCG
                               // style V - V_old (Eq. P_lobpcg, C = I), 2 none
  bool right_proj = true;      // projector before T (Table 3)
  // inner block GMRES (T = gm_steps steps on (A - sigma B) W = R, right-preconditioned
  // by the basic preconditioner prec)
  int gm_steps = 0;
  double2* gmV = nullptr;      // n x (gm_steps + 1) k, ld (gm_steps + 1) k: block Krylov basis
  double2 *gmT = nullptr, *gmAX = nullptr, *gmBX = nullptr;  // n x k
  double2* gmY = nullptr;      // gm_steps k x k: least-squares solution
  double2* h_gm = nullptr;     // pinned, per step: tracks C (3 trk) and R (3 k^2)
  int* h_gm_status = nullptr;  // pinned, per step: Cholesky status of its first pass
  double2* h_gmY = nullptr;    // pinned staging of gmY
  int64_t n_inner = 0;         // inner GMRES steps run
  double2* gram_part = nullptr;
  size_t gram_part_elems = 0;
  double* norm_part = nullptr;
  double* d_norms = nullptr;
  int* d_status = nullptr;    // [0..2] chol status of the passes of one orth call
  int* d_diag = nullptr;      // [0] shifted-Cholesky fallbacks, [1] Cholesky failures,
                              // [2] tensor-core waits that gave up
  bool tc = true;             // FP64 combinations on the tensor cores where supported
  int tc_wait_tries = gplhr::TC_WAIT_TRIES;  // limit of the tensor-core pipelines' waits
  bool tc_probe = false;      // test hook: combinations wait on a barrier nothing completes
  // pinned host staging
  double2* h_small = nullptr;  // coefficient uploads
  double2* h_phipsi = nullptr;
  double* h_norms = nullptr;
  int* h_diag = nullptr;
  // iteration state (host side)
  bool started = false;
  bool hasP = false;
  int q = 0, m = 0, it = 0;
  SqMat RA, RB, MA, MB;
  std::vector<double> resid;
  int64_t n_spmm = 0, n_prec = 0, n_qz = 0, n_launch = 0;
  int64_t h2d_bytes = 0, d2h_bytes = 0;  // host<->device traffic of the iteration
  // per-kernel-class accounting (always) and CUDA-event timing (when profiling)
  bool prof_on = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, int>> ev_rec;  // (class, start event index); stop = start + 1
  double k_flops[8] = {0}, k_bytes[8] = {0};
  int64_t k_launch[8] = {0};
  // CUDA graphs of an iteration's device segments (opts.graphs), keyed by the state
  // that fixes their launch sequence, with the accounting each replay adds
  struct Counters {
    double k_flops[8], k_bytes[8];
    int64_t k_launch[8], n_launch, n_spmm, n_prec, h2d, d2h;
  };
  struct SegGraph {
    cudaGraphExec_t exec;
    Counters delta;
  };
  bool graphs = false;
  std::map<uint64_t, SegGraph> seg_graphs;
  // SpMM launch shape per (group width G, columns per lane V): threads per CTA and the
  // grid cap in multiples of the SM count; the defaults, or the fastest candidate
  // measured at create time (opts.autotune)
  struct SpmmShape {
    int threads = 256, gridmul = 8;
    double us = 0.0;          // measured time of the chosen shape (autotune), microseconds
    double us_default = 0.0;  // measured time of the default shape 256 / 8
  };
  bool autotune = false;
  std::map<int, SpmmShape> spmm_shape;  // key 4 G + V
  const SpmmShape* spmm_force = nullptr;  // candidate being measured
  PkRecorder* rec = nullptr;  // non-null: device work is recorded, not issued
  // persistent batched iteration: recorded segments by segment key (a segment's launches
  // are fixed by its key, as for the CUDA graphs below), with the accounting each use adds;
  // rec_last is the recording of the segment just issued
  struct PkCached {
    PkRecorder rec;
    Counters delta;
  };
  std::map<uint64_t, PkCached>* pk_cache = nullptr;
  const PkRecorder* rec_last = nullptr;
  double2* pk_work = nullptr;  // 2 s_max^2 values: global work of a wide Cholesky (persistent batch)
  std::string err;
};

namespace {

#define CK(call)                                                                    \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      ctx->err = std::string(#call) + ": " + cudaGetErrorString(e_);                \
      return GPLHR_ECUDA;                                                           \
    }                                                                               \
  } while (0)

#define TRY(expr)                      \
  do {                                 \
    gplhr_status s_ = (expr);          \
    if (s_ != GPLHR_OK) return s_;     \
  } while (0)

const size_t kCombSmemMax = 200 * 1024;  // dynamic shared memory opted into per CTA
const double2 kOne = {1.0, 0.0};
const double2 kMinusOne = {-1.0, 0.0};

inline double2 d2(cd z) { return make_double2(z.real(), z.imag()); }

int grid_for(size_t work, int per_cta, int cap) {
  size_t g = (work + per_cta - 1) / per_cta;
  if (g < 1) g = 1;
  if (g > (size_t)cap) g = cap;
  return (int)g;
}

// ------------------------------------------------ recording (persistent mode) ----
// Record one launch (kind, gx x gy CTAs of 256 threads, smem bytes, arguments a).
template <class A>
void pk_rec(gplhr_ctx* ctx, int kind, int gx, int gy, size_t smem, const A& a) {
  PkRecorder* r = ctx->rec;
  const size_t off = (r->args.size() + 15) & ~(size_t)15;
  r->args.resize(off + sizeof(A));
  std::memcpy(r->args.data() + off, &a, sizeof(A));
  r->ops.push_back(PkRecorder::Op{kind, gx, gy, smem, off, sizeof(A)});
}

// An asynchronous copy on the context's stream, or, while recording: host-to-device
// before the segment's kernel, device-to-host after it, device-to-device as a step.
gplhr_status copy_async(gplhr_ctx* ctx, void* dst, const void* src, size_t bytes, cudaMemcpyKind kind) {
  if (ctx->rec) {
    if (kind == cudaMemcpyHostToDevice) {
      ctx->rec->pre.push_back(PkRecorder::Copy{dst, src, bytes});
    } else if (kind == cudaMemcpyDeviceToHost) {
      ctx->rec->post.push_back(PkRecorder::Copy{dst, src, bytes});
    } else {
      if (bytes % sizeof(double2) != 0) {
        ctx->err = "recorded device copy: size not a multiple of 16 bytes";
        return GPLHR_EINVAL;
      }
      const gplhr::PkBytes a{(const double2*)src, (double2*)dst, (int64_t)(bytes / sizeof(double2))};
      pk_rec(ctx, gplhr::PK_BYTES, grid_for(bytes / sizeof(double2), 256, 2 * ctx->num_sms), 1, 0, a);
    }
    return GPLHR_OK;
  }
  CK(cudaMemcpyAsync(dst, src, bytes, kind, ctx->stream));
  return GPLHR_OK;
}

// Block copy Y = X (n x w) and Y = alpha X1 + beta X2, launched or recorded.
void launch_copy_block(gplhr_ctx* ctx, int grid, int n, int w, const double2* X, int ldx, double2* Y, int ldy) {
  if (ctx->rec) {
    pk_rec(ctx, gplhr::PK_COPY_BLOCK, grid, 1, 0, gplhr::PkCopy{n, w, ldx, ldy, X, Y});
    return;
  }
  gplhr::copy_block_kernel<<<grid, 256, 0, ctx->stream>>>(n, w, X, ldx, Y, ldy);
}

void launch_axpby(gplhr_ctx* ctx, int grid, int n, int w, double2 alpha, const double2* X1, int ld1, double2 beta,
                  const double2* X2, int ld2, double2* Y, int ldy) {
  if (ctx->rec) {
    pk_rec(ctx, gplhr::PK_AXPBY, grid, 1, 0, gplhr::PkAxpby{n, w, ld1, ld2, ldy, alpha, beta, X1, X2, Y});
    return;
  }
  gplhr::axpby_kernel<<<grid, 256, 0, ctx->stream>>>(n, w, alpha, X1, ld1, beta, X2, ld2, Y, ldy);
}

// ----------------------------------------------------------- accounting ----
// Kernel classes for the per-class report (gplhr_profile_read).
enum { KC_SPMM = 0, KC_GRAM = 1, KC_COMBINE = 2, KC_PREC = 3, KC_CHOL = 4, KC_OTHER = 5, KC_GRAM_TC = 6,
       KC_COMBINE_TC = 7, KC_N = 8 };

// Opens a timed section of class c (one or more launches); returns its handle.
int prof_begin(gplhr_ctx* ctx, int c, double flops, double bytes, int launches = 1) {
  ctx->k_flops[c] += flops;
  ctx->k_bytes[c] += bytes;
  ctx->k_launch[c] += launches;
  ctx->n_launch += launches;
  if (!ctx->prof_on) return -1;
  const int idx = (int)ctx->ev_rec.size() * 2;
  while ((int)ctx->ev_pool.size() < idx + 2) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return -1;
    ctx->ev_pool.push_back(e);
  }
  cudaEventRecord(ctx->ev_pool[idx], ctx->stream);
  ctx->ev_rec.emplace_back(c, idx);
  return idx;
}
void prof_end(gplhr_ctx* ctx, int h) {
  if (h >= 0) cudaEventRecord(ctx->ev_pool[h + 1], ctx->stream);
}

gplhr_ctx::Counters snap_counters(const gplhr_ctx* ctx) {
  gplhr_ctx::Counters c;
  for (int i = 0; i < 8; ++i) {
    c.k_flops[i] = ctx->k_flops[i];
    c.k_bytes[i] = ctx->k_bytes[i];
    c.k_launch[i] = ctx->k_launch[i];
  }
  c.n_launch = ctx->n_launch;
  c.n_spmm = ctx->n_spmm;
  c.n_prec = ctx->n_prec;
  c.h2d = ctx->h2d_bytes;
  c.d2h = ctx->d2h_bytes;
  return c;
}

void restore_counters(gplhr_ctx* ctx, const gplhr_ctx::Counters& c) {
  for (int i = 0; i < 8; ++i) {
    ctx->k_flops[i] = c.k_flops[i];
    ctx->k_bytes[i] = c.k_bytes[i];
    ctx->k_launch[i] = c.k_launch[i];
  }
  ctx->n_launch = c.n_launch;
  ctx->n_spmm = c.n_spmm;
  ctx->n_prec = c.n_prec;
  ctx->h2d_bytes = c.h2d;
  ctx->d2h_bytes = c.d2h;
}

// Device work of one segment of an iteration (a run of launches and copies between two
// host round trips), issued by `issue` on the context's stream.  With opts.graphs the
// first run for a given key is captured into a CUDA graph, which later runs replay;
// every kernel argument of the segment must then be fixed by the key, and the small
// coefficient matrices reach the device through pinned staging buffers that the host
// fills before the segment runs (the graph's copies read them when it executes).
void add_counters(gplhr_ctx* ctx, const gplhr_ctx::Counters& d) {
  for (int i = 0; i < 8; ++i) {
    ctx->k_flops[i] += d.k_flops[i];
    ctx->k_bytes[i] += d.k_bytes[i];
    ctx->k_launch[i] += d.k_launch[i];
  }
  ctx->n_launch += d.n_launch;
  ctx->n_spmm += d.n_spmm;
  ctx->n_prec += d.n_prec;
  ctx->h2d_bytes += d.h2d;
  ctx->d2h_bytes += d.d2h;
}

gplhr_ctx::Counters diff_counters(const gplhr_ctx::Counters& c1, const gplhr_ctx::Counters& c0) {
  gplhr_ctx::Counters d;
  for (int i = 0; i < 8; ++i) {
    d.k_flops[i] = c1.k_flops[i] - c0.k_flops[i];
    d.k_bytes[i] = c1.k_bytes[i] - c0.k_bytes[i];
    d.k_launch[i] = c1.k_launch[i] - c0.k_launch[i];
  }
  d.n_launch = c1.n_launch - c0.n_launch;
  d.n_spmm = c1.n_spmm - c0.n_spmm;
  d.n_prec = c1.n_prec - c0.n_prec;
  d.h2d = c1.h2d - c0.h2d;
  d.d2h = c1.d2h - c0.d2h;
  return d;
}

gplhr_status run_segment(gplhr_ctx* ctx, uint64_t key, const std::function<gplhr_status()>& issue) {
  if (ctx->pk_cache) {  // persistent batch: record once per key, reuse the recording after
    auto it = ctx->pk_cache->find(key);
    if (it != ctx->pk_cache->end()) {
      add_counters(ctx, it->second.delta);
      ctx->rec_last = &it->second.rec;
      return GPLHR_OK;
    }
    const gplhr_ctx::Counters c0 = snap_counters(ctx);
    gplhr_ctx::PkCached& c = (*ctx->pk_cache)[key];
    c.rec.clear();
    ctx->rec = &c.rec;
    const gplhr_status st = issue();
    ctx->rec = nullptr;
    if (st != GPLHR_OK) {
      ctx->pk_cache->erase(key);
      return st;
    }
    c.delta = diff_counters(snap_counters(ctx), c0);
    ctx->rec_last = &c.rec;
    return GPLHR_OK;
  }
  if (ctx->rec || !ctx->graphs || ctx->prof_on || ctx->gm_steps > 0) return issue();
  auto it = ctx->seg_graphs.find(key);
  if (it != ctx->seg_graphs.end()) {
    CK(cudaGraphLaunch(it->second.exec, ctx->stream));
    const gplhr_ctx::Counters& d = it->second.delta;
    for (int i = 0; i < 8; ++i) {
      ctx->k_flops[i] += d.k_flops[i];
      ctx->k_bytes[i] += d.k_bytes[i];
      ctx->k_launch[i] += d.k_launch[i];
    }
    ctx->n_launch += d.n_launch;
    ctx->n_spmm += d.n_spmm;
    ctx->n_prec += d.n_prec;
    ctx->h2d_bytes += d.h2d;
    ctx->d2h_bytes += d.d2h;
    return GPLHR_OK;
  }
  const gplhr_ctx::Counters c0 = snap_counters(ctx);
  CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
  const gplhr_status st = issue();
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
  if (st != GPLHR_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    ctx->err = std::string("stream capture of an iteration segment: ") + cudaGetErrorString(e);
    return GPLHR_ECUDA;
  }
  cudaGraphExec_t ex = nullptr;
  const cudaError_t ei = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  CK(ei);
  const gplhr_ctx::Counters c1 = snap_counters(ctx);
  gplhr_ctx::Counters d;
  for (int i = 0; i < 8; ++i) {
    d.k_flops[i] = c1.k_flops[i] - c0.k_flops[i];
    d.k_bytes[i] = c1.k_bytes[i] - c0.k_bytes[i];
    d.k_launch[i] = c1.k_launch[i] - c0.k_launch[i];
  }
  d.n_launch = c1.n_launch - c0.n_launch;
  d.n_spmm = c1.n_spmm - c0.n_spmm;
  d.n_prec = c1.n_prec - c0.n_prec;
  d.h2d = c1.h2d - c0.h2d;
  d.d2h = c1.d2h - c0.d2h;
  ctx->seg_graphs[key] = gplhr_ctx::SegGraph{ex, d};
  CK(cudaGraphLaunch(ex, ctx->stream));  // the capture recorded the work; run it (counted once above)
  return GPLHR_OK;
}

// Key of a segment's launch sequence: segment id and the iteration state it depends on.
uint64_t seg_key(int seg, int q, int m, int kk, int s, int flags) {
  return (uint64_t)seg | ((uint64_t)(q & 0xFF) << 4) | ((uint64_t)(m & 0xFF) << 12) | ((uint64_t)(kk & 0xFF) << 20) |
         ((uint64_t)(s & 0xFFFF) << 28) | ((uint64_t)(flags & 0xFF) << 44);
}

// ------------------------------------------------------------------ launches --

gplhr_status launch_spmm_f64(gplhr_ctx* ctx, const DevCsr& M, const DevCsr* M2, Blk X, int w, Blk Y, Blk Y2);
gplhr_status launch_spmm_f32(gplhr_ctx* ctx, const DevCsr& M, const DevCsr* M2, Blk X, int w, Blk Y, Blk Y2);
gplhr_status launch_spmm_one(gplhr_ctx* ctx, const DevCsr& M, const DevCsr* M2, Blk X, int w, Blk Y, Blk Y2,
                             bool fp32 = false) {
  return fp32 ? launch_spmm_f32(ctx, M, M2, X, w, Y, Y2) : launch_spmm_f64(ctx, M, M2, X, w, Y, Y2);
}

// One launch of the row-group SpMM for a block of w <= 32 V columns: G lanes per row,
// the power of two >= ceil(w / V), at least 4.
template <typename T, int V, typename VTA, typename VTB>
void launch_spmm_g(gplhr_ctx* ctx, gplhr::CsrDev<VTA> a, gplhr::CsrDev<VTB> b, int hasB,
                   const gplhr::cplx<T>* X, int ldx, int w, double2* Y, int ldy, double2* Y2, int ldy2) {
  int G = 4;
  while (G * V < w) G <<= 1;
  gplhr_ctx::SpmmShape sh;
  if (ctx->spmm_force) {
    sh = *ctx->spmm_force;
  } else {
    const auto it = ctx->spmm_shape.find(4 * G + V);
    if (it != ctx->spmm_shape.end()) sh = it->second;
  }
  if (ctx->rec) sh = gplhr_ctx::SpmmShape{};  // the persistent kernel runs 256 threads per CTA
  const int rows_per_cta = (sh.threads / 32) * (32 / G);
  const int grid = grid_for((size_t)ctx->n, rows_per_cta, sh.gridmul * ctx->num_sms);
  const int nt = sh.threads;
  if (ctx->rec) {
    constexpr bool cpa = sizeof(VTA) == 2 * sizeof(T), cpb = sizeof(VTB) == 2 * sizeof(T);
    const int gi = G == 4 ? 0 : G == 8 ? 1 : G == 16 ? 2 : 3;
    const gplhr::PkSpmm o{ctx->n, hasB, ldx,    w,      ldy,   ldy2, a.rowptr, a.col, a.val,
                          b.rowptr, b.col, b.val, X, Y, Y2};
    pk_rec(ctx, gplhr::pk_spmm_code(V == 2 ? 1 : 0, cpa ? 1 : 0, cpb ? 1 : 0, gi), grid, 1, 0, o);
    return;
  }
  switch (G) {
    case 4:
      gplhr::spmm_kernel<VTA, VTB, T, 4, V><<<grid, nt, 0, ctx->stream>>>(ctx->n, a, b, hasB, X, ldx, w, Y, ldy, Y2, ldy2);
      break;
    case 8:
      gplhr::spmm_kernel<VTA, VTB, T, 8, V><<<grid, nt, 0, ctx->stream>>>(ctx->n, a, b, hasB, X, ldx, w, Y, ldy, Y2, ldy2);
      break;
    case 16:
      gplhr::spmm_kernel<VTA, VTB, T, 16, V><<<grid, nt, 0, ctx->stream>>>(ctx->n, a, b, hasB, X, ldx, w, Y, ldy, Y2,
                                                                         ldy2);
      break;
    default:
      gplhr::spmm_kernel<VTA, VTB, T, 32, V><<<grid, nt, 0, ctx->stream>>>(ctx->n, a, b, hasB, X, ldx, w, Y, ldy, Y2,
                                                                         ldy2);
      break;
  }
}

// Dispatch on the value types of M (and M2): real or complex values, stored as VR / VC.
template <typename T, int V, typename VR, typename VC>
void launch_spmm_types(gplhr_ctx* ctx, const DevCsr& M, const DevCsr* M2, const void* mval, const void* m2val,
                       const gplhr::cplx<T>* X, int ldx, int w, double2* Y, int ldy, double2* Y2, int ldy2) {
  gplhr::CsrDev<VR> ar{M.rowptr, M.col, (const VR*)mval};
  gplhr::CsrDev<VC> ac{M.rowptr, M.col, (const VC*)mval};
  if (!M2) {
    if (M.dtype == GPLHR_R64)
      launch_spmm_g<T, V>(ctx, ar, ar, 0, X, ldx, w, Y, ldy, nullptr, 0);
    else
      launch_spmm_g<T, V>(ctx, ac, ac, 0, X, ldx, w, Y, ldy, nullptr, 0);
    return;
  }
  gplhr::CsrDev<VR> br{M2->rowptr, M2->col, (const VR*)m2val};
  gplhr::CsrDev<VC> bc{M2->rowptr, M2->col, (const VC*)m2val};
  if (M.dtype == GPLHR_R64 && M2->dtype == GPLHR_R64)
    launch_spmm_g<T, V>(ctx, ar, br, 1, X, ldx, w, Y, ldy, Y2, ldy2);
  else if (M.dtype == GPLHR_R64)
    launch_spmm_g<T, V>(ctx, ar, bc, 1, X, ldx, w, Y, ldy, Y2, ldy2);
  else if (M2->dtype == GPLHR_R64)
    launch_spmm_g<T, V>(ctx, ac, br, 1, X, ldx, w, Y, ldy, Y2, ldy2);
  else
    launch_spmm_g<T, V>(ctx, ac, bc, 1, X, ldx, w, Y, ldy, Y2, ldy2);
}

// Algorithmic flops and bytes of one sparse product: values (vb bytes real, 2 vb
// complex) and int32 indices read once, row pointers once, the output written once
// (complex128).  The caller adds the reads of the input block.
void spmm_cost(gplhr_ctx* ctx, const DevCsr& D, int w, double vb, double& fl, double& by) {
  const bool cplx = D.dtype == GPLHR_C128;
  fl += (cplx ? 8.0 : 4.0) * (double)D.nnz * w;  // real x complex = 2 FMA
  by += (double)D.nnz * ((cplx ? 2.0 : 1.0) * vb + 4.0) + 4.0 * (ctx->n + 1.0) + 16.0 * ctx->n * w;
}

// FP32 sparse products: the input block is converted to complex64 once (the
// double -> float conversion runs on the FP64 pipe, and a gather touches each input
// row once per nonzero), into rows of even length (16-byte aligned for the two-column
// loads), and the matrix values come from their FP32 copies.
gplhr_status launch_spmm_f32(gplhr_ctx* ctx, const DevCsr& M, const DevCsr* M2, Blk X, int w, Blk Y, Blk Y2) {
  if (!M.val32 || (M2 && !M2->val32) || !ctx->X32 || w > ctx->k) return launch_spmm_f64(ctx, M, M2, X, w, Y, Y2);
  const int ld32 = (w + 1) & ~1;
  // the conversion reads 16 and writes 8 bytes per element; the products read 8
  double fl = 0.0, by = (16.0 + 8.0 + 8.0) * ctx->n * w;
  spmm_cost(ctx, M, w, 4.0, fl, by);
  if (M2) spmm_cost(ctx, *M2, w, 4.0, fl, by);
  const int ph = prof_begin(ctx, KC_SPMM, fl, by, 2);
  const int gconv = grid_for((size_t)ctx->n * w, 256, 8 * ctx->num_sms);
  if (ctx->rec)
    pk_rec(ctx, gplhr::PK_TO_C64, gconv, 1, 0, gplhr::PkToC64{ctx->n, w, X.ld, ld32, X.p, ctx->X32});
  else
    gplhr::to_c64_kernel<<<gconv, 256, 0, ctx->stream>>>(ctx->n, w, X.p, X.ld, ctx->X32, ld32);
  for (int c0 = 0; c0 < w; c0 += 64) {
    const int wc = std::min(64, w - c0);
    launch_spmm_types<float, 2, float, float2>(ctx, M, M2, M.val32, M2 ? M2->val32 : nullptr, ctx->X32 + c0, ld32,
                                               wc, Y.p + c0, Y.ld, M2 ? Y2.p + c0 : nullptr, Y2.ld);
  }
  prof_end(ctx, ph);
  CK(cudaGetLastError());
  return GPLHR_OK;
}

gplhr_status launch_spmm_f64(gplhr_ctx* ctx, const DevCsr& M, const DevCsr* M2, Blk X, int w, Blk Y, Blk Y2) {
  double fl = 0.0, by = 16.0 * ctx->n * w;  // the block, read once for both products
  spmm_cost(ctx, M, w, 8.0, fl, by);
  if (M2) spmm_cost(ctx, *M2, w, 8.0, fl, by);
  const int ph = prof_begin(ctx, KC_SPMM, fl, by, (w + 31) / 32);
  for (int c0 = 0; c0 < w; c0 += 32) {
    const int wc = std::min(32, w - c0);
    launch_spmm_types<double, 1, double, double2>(ctx, M, M2, M.val, M2 ? M2->val : nullptr, X.p + c0, X.ld, wc,
                                                  Y.p + c0, Y.ld, M2 ? Y2.p + c0 : nullptr, Y2.ld);
  }
  prof_end(ctx, ph);
  CK(cudaGetLastError());
  return GPLHR_OK;
}

// SpMM autotuner: for every group width G that the iteration's block widths 1..k
// select (in FP64, V = 1, and in the FP32 bulk phase, V = 2), time each launch shape
// (64, 128 or 256 threads per CTA; grid capped at 2, 4, 8, 16 or 64 CTAs per SM) on the
// context's own A (and B), 3 runs after a warm-up, CUDA events on its stream, and keep
// the fastest.  Every shape computes each row in the same lane group, so results do not
// depend on the choice.  The library's counters are left as they were.
gplhr_status autotune_spmm(gplhr_ctx* ctx) {
  const gplhr_ctx::Counters c0 = snap_counters(ctx);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  gplhr_status st = GPLHR_OK;
  const int threads[3] = {64, 128, 256}, gridmul[5] = {2, 4, 8, 16, 64};
  CK(cudaMemsetAsync(ctx->Z, 0, (size_t)ctx->n * ctx->s_max * sizeof(double2), ctx->stream));
  for (int V = 1; V <= (ctx->mixed ? 2 : 1) && st == GPLHR_OK; ++V) {
    for (int G = 4; G <= 32 && st == GPLHR_OK; G <<= 1) {
      const int wlo = G == 4 ? 1 : (G / 2) * V + 1;
      const int w = std::min(G * V, ctx->k);
      if (w < wlo) continue;
      gplhr_ctx::SpmmShape best;
      best.us = 1e30;
      for (int ti = 0; ti < 3 && st == GPLHR_OK; ++ti)
        for (int gi = 0; gi < 5 && st == GPLHR_OK; ++gi) {
          gplhr_ctx::SpmmShape cand;
          cand.threads = threads[ti];
          cand.gridmul = gridmul[gi];
          ctx->spmm_force = &cand;
          float ms = 0.0f;
          for (int rep = 0; rep < 4 && st == GPLHR_OK; ++rep) {
            if (rep == 1) cudaEventRecord(e0, ctx->stream);
            st = launch_spmm_one(ctx, ctx->A, ctx->hasB ? &ctx->B : nullptr, Blk{ctx->Z, ctx->s_max}, w,
                                 Blk{ctx->AZ, ctx->s_max}, Blk{ctx->hasB ? ctx->BZ : nullptr, ctx->s_max}, V == 2);
          }
          ctx->spmm_force = nullptr;
          if (st != GPLHR_OK) break;
          cudaEventRecord(e1, ctx->stream);
          if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            ctx->err = "SpMM autotuning: event timing failed";
            st = GPLHR_ECUDA;
            break;
          }
          const double us = 1e3 * ms / 3.0;
          if (cand.threads == 256 && cand.gridmul == 8) best.us_default = us;
          if (us < best.us) {
            const double ud = best.us_default;
            best = cand;
            best.us = us;
            best.us_default = ud;
          }
        }
      if (st == GPLHR_OK) ctx->spmm_shape[4 * G + V] = best;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  restore_counters(ctx, c0);
  return st;
}

gplhr_status project_out(gplhr_ctx* ctx, Blk L, int wl, Blk X, int w);

// Products with the pencil the iteration runs on: A X and (B != I) B X, or with a
// deflation basis (V1, Q1) the deflated maps (I - Q1 Q1^*) A (I - V1 V1^*) X and
// (I - Q1 Q1^*) B (I - V1 V1^*) X (Q1 = V1 when B = I).  X is projected in place.
gplhr_status pair_products(gplhr_ctx* ctx, Blk X, int w, Blk AX, Blk BX, bool fp32) {
  if (ctx->k1 > 0) TRY(project_out(ctx, Blk{ctx->dV1, ctx->k1}, ctx->k1, X, w));
  TRY(launch_spmm_one(ctx, ctx->A, ctx->hasB ? &ctx->B : nullptr, X, w, AX, BX, fp32));
  if (ctx->k1 > 0) {
    const Blk L{ctx->hasB ? ctx->dQ1 : ctx->dV1, ctx->k1};
    TRY(project_out(ctx, L, ctx->k1, AX, w));
    if (ctx->hasB) TRY(project_out(ctx, L, ctx->k1, BX, w));
  }
  return GPLHR_OK;
}

// AX = A X and (B != I) BX = B X (deflated pair when a deflation basis is set)
gplhr_status spmm_AB(gplhr_ctx* ctx, Blk X, int w, Blk AX, Blk BX) {
  if (w <= 0) return GPLHR_OK;
  ctx->n_spmm += 1;
  return pair_products(ctx, X, w, AX, BX, ctx->bulk32);
}

// C (wx x (wy0 + wy1), row-major) = X^* [Y0 Y1].  herm: X^* X (only the upper
// triangle is computed; the lower one is filled by conjugation).
template <int ACC>
void launch_gram_acc(gplhr_ctx* ctx, dim3 grid, size_t smem, int rows, Blk X, int wx, Blk Y0, int wy0,
                     Blk Y1, int wy1, int herm, int nout, int G, int RG, const int* skip, int mode) {
  if (ctx->rec) {
    const int lacc = ACC == 1 ? 0 : ACC == 2 ? 1 : ACC == 4 ? 2 : 3;
    const gplhr::PkGram o{ctx->n, rows, X.ld, wx,  Y0.ld, wy0, Y1.ld, wy1, herm, nout,
                          G,      RG,   X.p,  Y0.p, Y1.p, ctx->gram_part, skip};
    pk_rec(ctx, gplhr::PK_GRAM_BASE + 4 * mode + lacc, (int)grid.x, (int)grid.y, smem, o);
    return;
  }
  if (mode == 2)
    gplhr::gram_partial_x32_kernel<ACC><<<grid, gplhr::GRAM_THREADS, smem, ctx->stream>>>(
        ctx->n, rows, X.p, X.ld, wx, Y0.p, Y0.ld, wy0, Y1.p, Y1.ld, wy1, herm, nout, G, RG, ctx->gram_part, skip);
  else if (mode == 1)
    gplhr::gram_partial_kernel<ACC, float><<<grid, gplhr::GRAM_THREADS, smem, ctx->stream>>>(
        ctx->n, rows, X.p, X.ld, wx, Y0.p, Y0.ld, wy0, Y1.p, Y1.ld, wy1, herm, nout, G, RG, ctx->gram_part, skip);
  else
    gplhr::gram_partial_kernel<ACC, double><<<grid, gplhr::GRAM_THREADS, smem, ctx->stream>>>(
        ctx->n, rows, X.p, X.ld, wx, Y0.p, Y0.ld, wy0, Y1.p, Y1.ld, wy1, herm, nout, G, RG, ctx->gram_part, skip);
}

// fp32: FP32 arithmetic (projection coefficients in the bulk phase).  Otherwise an
// FP64-accurate Gram: DFMA, or in the bulk phase (FP32-valued blocks) exact products
// on the FP32 pipe with compensated accumulation (gram_partial_x32_kernel).
// FP64 Gram product on the tensor cores (tc.cuh): one persistent CTA per SM over 128-row
// windows, partials reduced deterministically.  Shapes: wx <= 128, wy <= 32, with the
// accumulators of all M tiles in tensor memory.
bool gram_tc_fits(const gplhr_ctx* ctx, int wx, int wy) {
  const int np = ((2 * wy + 15) / 16) * 16, mt = (2 * wx + 127) / 128;
  return ctx->tc && wx <= gplhr::TG_AMAX && wy <= gplhr::TG_BMAX && mt * gplhr::TC_DIAG * np <= 512 &&
         ctx->n >= 2048 && wx * wy >= 400 &&
         (size_t)std::min(ctx->num_sms, (ctx->n + gplhr::TG_WIN - 1) / gplhr::TG_WIN) * wx * wy <=
             ctx->gram_part_elems;
}

// cbw > 0: column blocks of cbw columns of [Y0 Y1], all in one launch (grid y = block),
// the SMs shared evenly between the blocks.
gplhr_status gram_tc(gplhr_ctx* ctx, Blk X, int wx, Blk Y0, int wy0, Blk Y1, int wy1, double2* C, const int* skip,
                     int nout_count, bool count, int ldc, int cbw = 0) {
  gplhr::TcGramArgs t{};
  const int wy = wy0 + wy1;
  if (cbw <= 0 || cbw > wy) cbw = wy;
  const int nblk = (wy + cbw - 1) / cbw;
  t.n = ctx->n;
  t.X = X.p;
  t.ldx = X.ld;
  t.wx = wx;
  t.Y0 = Y0.p;
  t.ldy0 = Y0.ld;
  t.wy0 = wy0;
  t.Y1 = Y1.p;
  t.ldy1 = Y1.ld;
  t.wy1 = wy1;
  t.partial = ctx->gram_part;
  t.skip = skip;
  t.err = ctx->d_diag + 2;
  t.wait_tries = ctx->tc_wait_tries;
  t.np = ((2 * cbw + 15) / 16) * 16;
  t.mt = (2 * wx + 127) / 128;
  t.cbw = cbw;
  t.tmem_cols = 32;
  while (t.tmem_cols < t.mt * gplhr::TC_DIAG * t.np) t.tmem_cols <<= 1;
  const int nwin = (ctx->n + gplhr::TG_WIN - 1) / gplhr::TG_WIN;
  const int grid = std::max(1, std::min(ctx->num_sms / nblk, nwin));
  const bool self = X.p == Y0.p && wy1 == 0;
  const double by = 16.0 * ctx->n * (self ? wx : wx + wy);
  const int ph = prof_begin(ctx, KC_GRAM_TC, count ? 8.0 * ctx->n * nout_count : 0.0, count ? by : 0.0, 1 + nblk);
  gplhr::tc_gram_kernel<<<dim3(grid, nblk), gplhr::TG_THREADS, gplhr::tg_smem_bytes(t.mt, t.np), ctx->stream>>>(t);
  CK(cudaGetLastError());
  for (int b = 0; b < nblk; ++b) {
    const int wyb = std::min(cbw, wy - b * cbw), nout = wx * wyb;
    gplhr::gram_reduce_kernel<<<(nout + gplhr::GRED_WARPS - 1) / gplhr::GRED_WARPS, 32 * gplhr::GRED_WARPS, 0,
                                 ctx->stream>>>(grid, nout, wx, wyb, 0, ctx->gram_part + (size_t)b * grid * wx * cbw,
                                                C + b * cbw, ldc, skip);
  }
  prof_end(ctx, ph);
  CK(cudaGetLastError());
  return GPLHR_OK;
}

// Narrow FP64 Gram products on the tensor cores (tc.cuh, tc_gram_narrow_kernel): digit
// planes stacked along M and N, one pipelined CTA per SM over 128-row windows.
struct TnShape {
  int mt, np, ts, cols;
  size_t smem;
};
bool gram_tn_fits(const gplhr_ctx* ctx, int wx, int wy, bool self, TnShape* sh = nullptr) {
  if (!ctx->tc || ctx->n < 2048 || wx < 1 || wy < 1 || wx > gplhr::TN_XMAX || wy > gplhr::TN_YMAX ||
      (self ? wx : wx + wy) > 4 * gplhr::TN_TASKS)
    return false;
  TnShape t;
  t.mt = (14 * wx + 127) / 128;
  t.np = ((2 * wy + 15) / 16) * 16;
  const int buf = t.mt * 7 * t.np;
  if (buf > 512) return false;
  t.ts = 2 * buf <= 512 ? 2 : 1;
  t.cols = 32;
  while (t.cols < t.ts * buf) t.cols <<= 1;
  t.smem = gplhr::tn_smem_bytes(t.mt, t.np, wx, wy);
  if (t.smem > kCombSmemMax) return false;
  if ((size_t)std::min(ctx->num_sms, (ctx->n + gplhr::TN_HALF - 1) / gplhr::TN_HALF) * wx * wy >
      ctx->gram_part_elems)
    return false;
  if (sh) *sh = t;
  return true;
}

// trans: X and Y0 were swapped by the caller (C = (Y0^* X)^*), the reduction writes C.
gplhr_status gram_tn(gplhr_ctx* ctx, Blk X, int wx, Blk Y0, int wy0, Blk Y1, int wy1, double2* C, const int* skip,
                     int nout_count, bool count, bool self, const TnShape& sh, int ldc, bool trans = false) {
  gplhr::TcGramNArgs t{};
  const int wy = wy0 + wy1;
  t.n = ctx->n;
  t.X = X.p;
  t.ldx = X.ld;
  t.wx = wx;
  t.Y0 = Y0.p;
  t.ldy0 = Y0.ld;
  t.wy0 = wy0;
  t.Y1 = Y1.p;
  t.ldy1 = Y1.ld;
  t.wy1 = wy1;
  t.self = self ? 1 : 0;
  t.partial = ctx->gram_part;
  t.skip = skip;
  t.err = ctx->d_diag + 2;
  t.wait_tries = ctx->tc_wait_tries;
  t.mt = sh.mt;
  t.np = sh.np;
  t.ts = sh.ts;
  t.tmem_cols = sh.cols;
  const int grid = std::min(ctx->num_sms, (ctx->n + gplhr::TN_HALF - 1) / gplhr::TN_HALF);
  const double by = 16.0 * ctx->n * (self ? wx : wx + wy);
  const int ph = prof_begin(ctx, KC_GRAM_TC, count ? 8.0 * ctx->n * nout_count : 0.0, count ? by : 0.0, 2);
  if ((self ? wx : wx + wy) <= 16)
    gplhr::tc_gram_narrow_kernel<4><<<grid, gplhr::TN_THREADS, sh.smem, ctx->stream>>>(t);
  else
    gplhr::tc_gram_narrow_kernel<8><<<grid, gplhr::TN_THREADS, sh.smem, ctx->stream>>>(t);
  CK(cudaGetLastError());
  const int nout = wx * wy;
  gplhr::gram_reduce_kernel<<<(nout + gplhr::GRED_WARPS - 1) / gplhr::GRED_WARPS, 32 * gplhr::GRED_WARPS, 0,
                               ctx->stream>>>(grid, nout, wx, wy, trans ? 2 : 0, ctx->gram_part, C, ldc, skip);
  prof_end(ctx, ph);
  CK(cudaGetLastError());
  return GPLHR_OK;
}

// Wide FP64 Gram products on the tensor cores (tc.cuh, tc_gram_wide_kernel): wx <= 64,
// wy <= 32, one pipelined CTA per SM over 128-row windows.
const size_t kTwSmemMax = 212 * 1024;  // dynamic shared memory opted into by the wide Gram
bool gram_tw_fits(const gplhr_ctx* ctx, int wx, int wy, bool self) {
  if (!ctx->tc || ctx->n < 2048 || wx < 1 || wy < 1 || wx > gplhr::TW_XMAX || wy > gplhr::TW_YMAX ||
      wx * wy < 128)
    return false;
  const int np = ((2 * wy + 15) / 16) * 16;
  if (gplhr::tw_smem_bytes(np, wx, wy) > kTwSmemMax) return false;
  (void)self;
  return (size_t)std::min(ctx->num_sms, (ctx->n + gplhr::TW_WIN - 1) / gplhr::TW_WIN) * wx * wy <=
         ctx->gram_part_elems;
}

// trans: X and Y0 were swapped by the caller (C = (Y0^* X)^*), the reduction writes C.
gplhr_status gram_tw(gplhr_ctx* ctx, Blk X, int wx, Blk Y0, int wy0, Blk Y1, int wy1, double2* C, const int* skip,
                     int nout_count, bool count, bool self, int ldc, bool trans = false) {
  gplhr::TcGramWArgs t{};
  const int wy = wy0 + wy1;
  t.n = ctx->n;
  t.X = X.p;
  t.ldx = X.ld;
  t.wx = wx;
  t.Y0 = Y0.p;
  t.ldy0 = Y0.ld;
  t.wy0 = wy0;
  t.Y1 = Y1.p;
  t.ldy1 = Y1.ld;
  t.wy1 = wy1;
  t.self = self ? 1 : 0;
  t.partial = ctx->gram_part;
  t.skip = skip;
  t.err = ctx->d_diag + 2;
  t.wait_tries = ctx->tc_wait_tries;
  t.np = ((2 * wy + 15) / 16) * 16;
  t.ts = 2 * gplhr::TC_DIAG * t.np <= 512 ? 2 : 1;
  t.tmem_cols = 32;
  while (t.tmem_cols < t.ts * gplhr::TC_DIAG * t.np) t.tmem_cols <<= 1;
  const int nwin = (ctx->n + gplhr::TW_WIN - 1) / gplhr::TW_WIN;
  const int grid = std::min(ctx->num_sms, nwin);
  const double by = 16.0 * ctx->n * (self ? wx : wx + wy);
  const int ph = prof_begin(ctx, KC_GRAM_TC, count ? 8.0 * ctx->n * nout_count : 0.0, count ? by : 0.0, 2);
  gplhr::tc_gram_wide_kernel<<<grid, gplhr::TW_THREADS, gplhr::tw_smem_bytes(t.np, wx, wy), ctx->stream>>>(t);
  CK(cudaGetLastError());
  const int nout = wx * wy;
  gplhr::gram_reduce_kernel<<<(nout + gplhr::GRED_WARPS - 1) / gplhr::GRED_WARPS, 32 * gplhr::GRED_WARPS, 0,
                               ctx->stream>>>(grid, nout, wx, wy, trans ? 2 : 0, ctx->gram_part, C, ldc, skip);
  prof_end(ctx, ph);
  CK(cudaGetLastError());
  return GPLHR_OK;
}

// C (wx x wy, row stride ldc, wy when ldc < 0) = X^* [Y0 Y1].  The FP64 product (mode 0)
// goes to the tensor cores when a form fits: narrow, narrow transposed, wide, wide
// transposed, serial; a product with more than 32 columns of [Y0 Y1] is computed in
// column blocks of at most 32, each into its columns of C; else DFMA.
gplhr_status gram(gplhr_ctx* ctx, Blk X, int wx, Blk Y0, int wy0, Blk Y1, int wy1, double2* C,
                  const int* skip = nullptr, bool herm = false, bool count = true, bool fp32 = false,
                  int force_mode = -1, int ldc = -1) {
  const int mode = force_mode >= 0 ? force_mode : (fp32 ? 1 : (ctx->bulk32 ? 2 : 0));
  const int wy = wy0 + wy1;
  if (ldc < 0) ldc = wy;
  const bool self = X.p == Y0.p && X.ld == Y0.ld && wy0 == wx && wy1 == 0;
  const bool tcok = mode == 0 && force_mode < 0;
  TnShape tn;
  // (a Hermitian request gets the full product on the tensor cores; the algorithmic count
  // stays the half)
  const int nout_tc = herm && self ? wx * (wx + 1) / 2 : wx * wy;
  if (tcok && gram_tn_fits(ctx, wx, wy, self, &tn))
    return gram_tn(ctx, X, wx, Y0, wy0, Y1, wy1, C, skip, nout_tc, count, self, tn, ldc);
  if (tcok && wy1 == 0 && !self && gram_tn_fits(ctx, wy0, wx, false, &tn))
    return gram_tn(ctx, Y0, wy0, X, wx, Blk{nullptr, 0}, 0, C, skip, wx * wy, count, false, tn, ldc, true);
  if (tcok && gram_tw_fits(ctx, wx, wy, self))
    return gram_tw(ctx, X, wx, Y0, wy0, Y1, wy1, C, skip, nout_tc, count, self, ldc);
  if (tcok && wy1 == 0 && !self && gram_tw_fits(ctx, wy0, wx, false))
    return gram_tw(ctx, Y0, wy0, X, wx, Blk{nullptr, 0}, 0, C, skip, wx * wy, count, false, ldc, true);
  if (tcok && gram_tc_fits(ctx, wx, wy))
    return gram_tc(ctx, X, wx, Y0, wy0, Y1, wy1, C, skip, nout_tc, count, ldc);
  if (tcok && ctx->tc && ctx->n >= 2048) {
    // outside the forms' shapes (wx <= 128): blocks, each a tensor-core product into its part
    // of C (the whole product's algorithmic work is booked here, the blocks' launches and
    // times with each block).  Three plans, by a cost per column read that was measured
    // on one GB300 at n = 65536 (narrow and wide forms ~1.9 us, the serial form with its
    // column blocks in one launch ~2.5 us):
    //   A: column blocks of [Y0 Y1] of the widest of 32, 24, 16, 8 columns that the narrow
    //      or wide form takes with all of X;
    //   B: column blocks of 32, 16 or 8 columns by the serial form, in one launch;
    //   C: X in two halves (wx > 64), each planned alike.
    auto plan_a = [&](int ax, int& cbw) {
      for (int cand : {32, 24, 16, 8}) {
        const int w = std::min(cand, wy);
        if (gram_tn_fits(ctx, ax, w, false) || gram_tw_fits(ctx, ax, w, false)) {
          cbw = w;
          const int nb = (wy + w - 1) / w;
          return 1.9 * (nb * ax + wy);
        }
      }
      cbw = 0;
      return 1e30;
    };
    auto plan_b = [&](int ax, int& cbw) {
      for (int cand : {32, 16, 8}) {
        const int w = std::min(cand, wy);
        if (gram_tc_fits(ctx, ax, w) && (size_t)ctx->num_sms * ax * w <= ctx->gram_part_elems) {
          cbw = w;
          const int nb = (wy + w - 1) / w;
          return 2.5 * (nb * ax + wy);
        }
      }
      cbw = 0;
      return 1e30;
    };
    int cba = 0, cbb = 0, tmp = 0;
    const double ca = plan_a(wx, cba), cb_cost = plan_b(wx, cbb);
    double cc = 1e30;
    const int xa = (wx + 1) / 2;
    if (wx > gplhr::TW_XMAX)
      cc = std::min(plan_a(xa, tmp), plan_b(xa, tmp)) + std::min(plan_a(wx - xa, tmp), plan_b(wx - xa, tmp));
    if (cc < ca && cc < cb_cost) {
      if (count) {
        ctx->k_flops[KC_GRAM_TC] += 8.0 * ctx->n * nout_tc;
        ctx->k_bytes[KC_GRAM_TC] += 16.0 * ctx->n * (self ? wx : wx + wy);
      }
      TRY(gram(ctx, X, xa, Y0, wy0, Y1, wy1, C, skip, false, false, fp32, -1, ldc));
      return gram(ctx, Blk{X.p + xa, X.ld}, wx - xa, Y0, wy0, Y1, wy1, C + (size_t)xa * ldc, skip, false, false,
                  fp32, -1, ldc);
    }
    if (cbb > 0 && cbb < wy && cb_cost <= ca)
      return gram_tc(ctx, X, wx, Y0, wy0, Y1, wy1, C, skip, nout_tc, count, ldc, cbb);
    const int cb = cba;
    if (cb > 0 && cb < wy) {
      if (count) {
        ctx->k_flops[KC_GRAM_TC] += 8.0 * ctx->n * nout_tc;
        ctx->k_bytes[KC_GRAM_TC] += 16.0 * ctx->n * (self ? wx : wx + wy);
      }
      for (int c0 = 0; c0 < wy; c0 += cb) {
        const int c1 = std::min(wy, c0 + cb);
        // the block's columns of Y0, then of Y1 (either part may be empty)
        const int a0 = std::min(c0, wy0), a1 = std::min(c1, wy0);
        const int e0 = std::max(c0, wy0) - wy0, e1 = std::max(c1, wy0) - wy0;
        Blk p0{Y0.p + a0, Y0.ld}, p1{e1 > e0 ? Y1.p + e0 : nullptr, Y1.ld};
        int n0 = a1 - a0, n1 = e1 - e0;
        if (n0 == 0) {
          p0 = p1;
          n0 = n1;
          p1 = Blk{nullptr, 0};
          n1 = 0;
        }
        TRY(gram(ctx, X, wx, p0, n0, p1, n1, C + c0, skip, false, false, fp32, -1, ldc));
      }
      return GPLHR_OK;
    }
  }
  if (herm && (wy1 != 0 || wy0 != wx)) herm = false;
  const int nout = herm ? wx * (wx + 1) / 2 : wx * wy;
  if (nout == 0) return GPLHR_OK;
  // accumulators per thread and output groups per CTA tile
  int acc = 8;
  while (acc > 1 && (nout + acc - 1) / acc < 128) acc >>= 1;
  const int groups = (nout + acc - 1) / acc;
  const int G = std::min(groups, gplhr::GRAM_THREADS);
  const int RG = gplhr::GRAM_THREADS / G;
  const int ntile = (groups + G - 1) / G;
  int nchunk = std::max(1, (4 * ctx->num_sms) / ntile);
  nchunk = std::min(nchunk, std::max(1, (ctx->n + gplhr::GRAM_ROWS - 1) / gplhr::GRAM_ROWS));
  while ((size_t)nchunk * nout > ctx->gram_part_elems && nchunk > 1) nchunk /= 2;
  int rows = (ctx->n + nchunk - 1) / nchunk;
  rows = ((rows + gplhr::GRAM_ROWS - 1) / gplhr::GRAM_ROWS) * gplhr::GRAM_ROWS;
  nchunk = (ctx->n + rows - 1) / rows;
  dim3 grid(nchunk, ntile);
  const size_t smem = mode == 2 ? std::max((size_t)gplhr::X32_ROWS * (wx + wy) * sizeof(float2),
                                           (size_t)RG * G * acc * sizeof(double2))
                                : std::max((size_t)gplhr::GRAM_ROWS * (wx + wy), (size_t)RG * G * acc) *
                                      sizeof(double2);
  const double by = 16.0 * ctx->n * (self ? wx : wx + wy);
  const int ph = prof_begin(ctx, KC_GRAM, count ? 8.0 * ctx->n * nout : 0.0, count ? by : 0.0, 2);
  switch (acc) {
    case 8: launch_gram_acc<8>(ctx, grid, smem, rows, X, wx, Y0, wy0, Y1, wy1, herm, nout, G, RG, skip, mode); break;
    case 4: launch_gram_acc<4>(ctx, grid, smem, rows, X, wx, Y0, wy0, Y1, wy1, herm, nout, G, RG, skip, mode); break;
    case 2: launch_gram_acc<2>(ctx, grid, smem, rows, X, wx, Y0, wy0, Y1, wy1, herm, nout, G, RG, skip, mode); break;
    default: launch_gram_acc<1>(ctx, grid, smem, rows, X, wx, Y0, wy0, Y1, wy1, herm, nout, G, RG, skip, mode); break;
  }
  CK(cudaGetLastError());
  const int gred = (nout + gplhr::GRED_WARPS - 1) / gplhr::GRED_WARPS;
  if (ctx->rec)
    pk_rec(ctx, gplhr::PK_GRAM_REDUCE, gred, 1, 0,
           gplhr::PkGramRed{nchunk, nout, wx, wy, herm ? 1 : 0, ldc, ctx->gram_part, C, skip});
  else
    gplhr::gram_reduce_kernel<<<gred, 32 * gplhr::GRED_WARPS, 0, ctx->stream>>>(nchunk, nout, wx, wy, herm ? 1 : 0,
                                                                                ctx->gram_part, C, ldc, skip);
  prof_end(ctx, ph);
  CK(cudaGetLastError());
  return GPLHR_OK;
}

struct In {
  Blk X;
  int w;
  const double2* C;  // w x c; row stride ldc (0: c)
  double2 alpha;
  int ldc = 0;
};

// The combination on the tensor cores (FP64 by integer digits, tc.cuh): one persistent
// pipelined CTA per SM, 128 rows per tile; two digit stages and two accumulator buffers
// where shared and tensor memory allow.
gplhr_status combine_tc(gplhr_ctx* ctx, gplhr::CombArgs a, int wsum, int c, int c_store, double flops,
                        double bytes) {
  gplhr::TcCombArgs t{};
  t.a = a;
  t.a.upper = 0;
  t.kp = ((2 * wsum + 15) / 16) * 16;
  t.np = ((2 * c + 15) / 16) * 16;
  t.ds = gplhr::tc_comb_smem_bytes(t.kp, t.np, 2) <= kCombSmemMax ? 2 : 1;
  t.ts = 2 * gplhr::TC_DIAG * t.np <= 512 ? 2 : 1;
  t.probe = ctx->tc_probe ? 1 : 0;
  t.tmem_cols = 32;
  while (t.tmem_cols < t.ts * gplhr::TC_DIAG * t.np) t.tmem_cols <<= 1;
  t.err = ctx->d_diag + 2;
  t.wait_tries = ctx->tc_wait_tries;
  const int ntiles = (ctx->n + gplhr::TC_ROWS - 1) / gplhr::TC_ROWS;
  // two CTAs per SM at K' <= 32, N' = 16 (both fit in shared and tensor memory; at K' = 32
  // with one digit stage each)
  const bool two = t.kp <= 32 && t.np == 16 && t.ts * gplhr::TC_DIAG * t.np <= 256;
  if (two && t.kp == 32) t.ds = 1;
  const int grid = std::min(ntiles, (two ? 2 : 1) * ctx->num_sms);
  const size_t smem = gplhr::tc_comb_smem_bytes(t.kp, t.np, t.ds);
  t.a.normpart = c_store < c ? ctx->norm_part : nullptr;
  const int ph = prof_begin(ctx, KC_COMBINE_TC, flops, bytes, c_store < c ? 2 : 1);
  switch (t.kp / 8) {
    case 2:
      if (two)
        gplhr::tc_combine_kernel<2, 2><<<grid, gplhr::TC_PIPE_THREADS, smem, ctx->stream>>>(ctx->n, t);
      else
        gplhr::tc_combine_kernel<2><<<grid, gplhr::TC_PIPE_THREADS, smem, ctx->stream>>>(ctx->n, t);
      break;
    case 4:
      if (two)
        gplhr::tc_combine_kernel<4, 2><<<grid, gplhr::TC_PIPE_THREADS, smem, ctx->stream>>>(ctx->n, t);
      else
        gplhr::tc_combine_kernel<4><<<grid, gplhr::TC_PIPE_THREADS, smem, ctx->stream>>>(ctx->n, t);
      break;
    case 6: gplhr::tc_combine_kernel<6><<<grid, gplhr::TC_PIPE_THREADS, smem, ctx->stream>>>(ctx->n, t); break;
    default: gplhr::tc_combine_kernel<8><<<grid, gplhr::TC_PIPE_THREADS, smem, ctx->stream>>>(ctx->n, t); break;
  }
  CK(cudaGetLastError());
  if (c_store < c) {
    const int nc = c - c_store;
    gplhr::norm_reduce_kernel<<<(nc + 3) / 4, 128, 0, ctx->stream>>>(grid, nc, ctx->norm_part, ctx->d_norms);
    CK(cudaGetLastError());
  }
  prof_end(ctx, ph);
  return GPLHR_OK;
}

// A combination wider than one tensor-core tile (more than 32 input or output columns)
// as several tensor-core launches: output column blocks of at most 32 columns, each the
// sum over chunks of at most 32 input columns; the first chunk of a block stores (beta as
// given), the later ones add to it (beta = 1).  Every launch rounds once, so a block
// carries one rounding per chunk, as a blocked FP64 sum does.  In place (outputs written
// over input columns) the order keeps the inputs of every launch intact: the one block
// that writes over inputs runs last, its chunk holding those inputs first; with upper
// (X <- X R^{-1}, R^{-1} upper triangular) the blocks run from the last to the first, and
// block [c0, c1) reads input columns 0 .. c1 - 1 only, its own chunk first.  Returns false,
// launching nothing, for shapes it does not cover (norm-only columns, outputs overlapping
// inputs in another pattern, more than COMB_MAX_IN pieces).  flops and bytes: the whole
// combination's algorithmic counts, booked with its first launch.
bool combine_tc_tiled(gplhr_ctx* ctx, const std::vector<In>& ins, Blk Y, int c, bool beta_one, const int* skip,
                      Blk Y2, int c_split, bool upper, double flops, double bytes, gplhr_status* st) {
  constexpr int KW = gplhr::TC_KMAX / 2, NW = gplhr::TC_NMAX / 2;
  const int nin = (int)ins.size();
  const int64_t n = ctx->n;
  // the input column (t, j) that output column o overwrites, if any
  std::vector<int> at(c, -1), aj(c, -1);
  for (int o = 0; o < c; ++o) {
    const double2* d = o < c_split ? Y.p + o : Y2.p + (o - c_split);
    const int ld = o < c_split ? Y.ld : Y2.ld;
    for (int t = 0; t < nin; ++t) {
      const double2* x = ins[t].X.p;
      const int lx = ins[t].X.ld, w = ins[t].w;
      const bool meet = d < x + (n - 1) * lx + w && x < d + (n - 1) * ld + 1;
      if (!meet) continue;
      const int64_t diff = d - x;
      if (ld != lx || diff < 0 || diff >= w) {
        // same rows, other columns of one buffer: no overlap; anything else is not covered
        if (ld == lx && ((diff % lx) + lx) % lx >= w && diff > -lx && diff < lx) continue;
        return false;
      }
      if (at[o] >= 0) return false;
      at[o] = t;
      aj[o] = (int)diff;
    }
  }
  struct Piece {
    int t, j0, j1;
  };
  const int nbo = (c + NW - 1) / NW;
  std::vector<int> cb(nbo + 1);
  for (int b = 0; b <= nbo; ++b) cb[b] = (int)((int64_t)c * b / nbo);
  // per block: the ordered list of launches, each a list of pieces of input columns
  std::vector<std::vector<std::vector<Piece>>> plan(nbo);
  auto pack = [&](std::vector<std::vector<Piece>>& L, int t, int j0, int j1) {
    while (j0 < j1) {
      int used = 0;
      if (!L.empty())
        for (const Piece& p : L.back()) used += p.j1 - p.j0;
      if (L.empty() || used >= KW || (int)L.back().size() >= gplhr::COMB_MAX_IN) {
        L.emplace_back();
        used = 0;
      }
      const int e = std::min(j1, j0 + KW - used);
      L.back().push_back(Piece{t, j0, e});
      j0 = e;
    }
  };
  std::vector<int> order(nbo);
  if (upper) {
    if (nin != 1 || ins[0].w != c || c_split != c) return false;
    for (int o = 0; o < c; ++o)
      if (at[o] >= 0 && aj[o] != o) return false;  // in place means Y = X
    for (int b = 0; b < nbo; ++b) {
      order[b] = nbo - 1 - b;
      plan[b].push_back({Piece{0, cb[b], cb[b + 1]}});
      plan[b].emplace_back();
      pack(plan[b], 0, 0, cb[b]);
      if (plan[b].back().empty()) plan[b].pop_back();
    }
  } else {
    int ab = -1;  // the one block that writes over inputs
    for (int o = 0; o < c; ++o)
      if (at[o] >= 0) {
        int b = 0;
        while (cb[b + 1] <= o) ++b;
        if (ab >= 0 && ab != b) return false;
        ab = b;
      }
    for (int b = 0, i = 0; b < nbo; ++b)
      if (b != ab) order[i++] = b;
    if (ab >= 0) order[nbo - 1] = ab;
    for (int b = 0; b < nbo; ++b) {
      if (b == ab) {  // first launch: the overwritten input columns of each input
        std::vector<int> lo(nin, INT32_MAX), hi(nin, -1);
        for (int o = cb[b]; o < cb[b + 1]; ++o)
          if (at[o] >= 0) {
            lo[at[o]] = std::min(lo[at[o]], aj[o]);
            hi[at[o]] = std::max(hi[at[o]], aj[o]);
          }
        std::vector<Piece> first;
        int wfirst = 0;
        for (int t = 0; t < nin; ++t)
          if (hi[t] >= 0) {
            first.push_back(Piece{t, lo[t], hi[t] + 1});
            wfirst += hi[t] + 1 - lo[t];
          }
        if (wfirst > KW) return false;
        plan[b].push_back(first);
        plan[b].emplace_back();
        for (int t = 0; t < nin; ++t) {
          if (hi[t] < 0) {
            pack(plan[b], t, 0, ins[t].w);
          } else {
            pack(plan[b], t, 0, lo[t]);
            pack(plan[b], t, hi[t] + 1, ins[t].w);
          }
        }
        if (plan[b].back().empty()) plan[b].pop_back();
      } else {
        for (int t = 0; t < nin; ++t) pack(plan[b], t, 0, ins[t].w);
      }
    }
  }
  bool first_launch = true;
  for (int i = 0; i < nbo; ++i) {
    const int b = order[i], c0 = cb[b], c1 = cb[b + 1], bw = c1 - c0;
    for (size_t l = 0; l < plan[b].size(); ++l) {
      gplhr::CombArgs a{};
      a.nin = (int)plan[b][l].size();
      int wsum = 0;
      for (int q = 0; q < a.nin; ++q) {
        const Piece& p = plan[b][l][q];
        const In& in = ins[p.t];
        const int ldc = in.ldc > 0 ? in.ldc : c;
        a.in[q] = gplhr::CombIn{in.X.p + p.j0, in.X.ld, p.j1 - p.j0, in.C + (size_t)p.j0 * ldc + c0, ldc, in.alpha};
        wsum += p.j1 - p.j0;
      }
      const int split = std::min(std::max(c_split - c0, 0), bw);
      a.Y = split > 0 ? Y.p + c0 : nullptr;
      a.ldy = Y.ld;
      a.Y2 = split < bw ? Y2.p + std::max(c0 - c_split, 0) : nullptr;
      a.ldy2 = Y2.ld;
      a.c = bw;
      a.c_split = split;
      a.c_store = bw;
      a.beta_one = (l > 0 || beta_one) ? 1 : 0;
      a.skip = skip;
      a.upper = 0;
      *st = combine_tc(ctx, a, wsum, bw, bw, first_launch ? flops : 0.0, first_launch ? bytes : 0.0);
      first_launch = false;
      if (*st != GPLHR_OK) return true;
    }
  }
  return true;
}

// Y(cols 0..c_split) / Y2 (cols c_split..c_store) = beta Y + sum alpha_t X_t C_t;
// columns c_store..c only contribute |.|^2 sums (reduced into ctx->d_norms).
gplhr_status combine(gplhr_ctx* ctx, const std::vector<In>& ins, Blk Y, int c, bool beta_one,
                     const int* skip = nullptr, Blk Y2 = Blk{nullptr, 0}, int c_split = -1,
                     int c_store = -1, bool count = true, int fp32 = -1, bool upper = false) {
  // fp32 = -1: the current phase decides (FP32 in the bulk phase of the mixed mode)
  const bool use32 = fp32 < 0 ? ctx->bulk32 : fp32 != 0;
  if (c <= 0 || ctx->n == 0) return GPLHR_OK;
  if (c_store < 0) c_store = c;
  if (c_split < 0) c_split = c_store;
  gplhr::CombArgs a{};
  a.nin = (int)ins.size();
  int wsum = 0;
  for (int t = 0; t < a.nin; ++t) {
    a.in[t] = gplhr::CombIn{ins[t].X.p, ins[t].X.ld, ins[t].w, ins[t].C, ins[t].ldc > 0 ? ins[t].ldc : c,
                            ins[t].alpha};
    wsum += ins[t].w;
  }
  a.Y = Y.p;
  a.ldy = Y.ld;
  a.Y2 = Y2.p;
  a.ldy2 = Y2.ld;
  a.c = c;
  a.c_split = c_split;
  a.c_store = c_store;
  a.beta_one = beta_one ? 1 : 0;
  a.skip = skip;
  a.upper = (upper && !use32 && a.nin == 1 && ins[0].w == c && c_store == c && c_split == c) ? 1 : 0;
  if (!use32 && ctx->tc && ctx->n >= 4 * gplhr::TC_ROWS) {
    const double fl = count ? 8.0 * ctx->n * (double)wsum * c : 0.0;
    const double by = count ? 16.0 * ctx->n * (wsum + c_store * (beta_one ? 2.0 : 1.0)) : 0.0;
    if (wsum <= gplhr::TC_KMAX / 2 && c <= gplhr::TC_NMAX / 2) return combine_tc(ctx, a, wsum, c, c_store, fl, by);
    gplhr_status st = GPLHR_OK;
    if (c_store == c && combine_tc_tiled(ctx, ins, Y, c, beta_one, skip, Y2, c_split, upper, fl, by, &st))
      return st;
  }
  int rows_tile = gplhr::comb_rows_tile(c, a.upper);
  const size_t esz = use32 ? sizeof(float2) : sizeof(double2);
  auto smem_of = [&](int rt) { return (size_t)(wsum * c + rt * wsum + rt * c) * esz; };
  // FP32 arithmetic is cheap next to the row loads: tiles of up to 4 outputs per thread
  // keep more loads in flight between the tile's two barriers (each output's sum is the
  // same, in the same order, whatever the tile)
  if (use32 && !a.upper)
    for (int f = 4; f > 1; f /= 2)
      if (smem_of(f * rows_tile) <= 48 * 1024) {
        rows_tile *= f;
        break;
      }
  while (!a.upper && rows_tile > 1 && smem_of(rows_tile) > kCombSmemMax) rows_tile /= 2;
  if (smem_of(rows_tile) > kCombSmemMax) {
    ctx->err = "combine: coefficient block too large for shared memory";
    return GPLHR_EINVAL;
  }
  a.rows_tile = rows_tile;
  const int grid = grid_for((size_t)ctx->n, std::max(rows_tile, 64), 4 * ctx->num_sms);
  const int rows_per_cta = (ctx->n + grid - 1) / grid;
  a.normpart = c_store < c ? ctx->norm_part : nullptr;
  const size_t smem = smem_of(rows_tile);
  double by = 16.0 * ctx->n * (wsum + c_store * (beta_one ? 2.0 : 1.0));
  const double macs = a.upper ? 0.5 * c * (c + 1.0) : (double)wsum * c;
  const int ph = prof_begin(ctx, KC_COMBINE, count ? 8.0 * ctx->n * macs : 0.0, count ? by : 0.0,
                           c_store < c ? 2 : 1);
  if (ctx->rec) {
    pk_rec(ctx, use32 ? gplhr::PK_COMBINE_F : gplhr::PK_COMBINE_D, grid, 1, smem, gplhr::PkComb{ctx->n, rows_per_cta, a});
    if (c_store < c) {
      const int nc = c - c_store;
      pk_rec(ctx, gplhr::PK_NORM_REDUCE, (nc + 7) / 8, 1, 0, gplhr::PkNormRed{grid, nc, ctx->norm_part, ctx->d_norms});
    }
    prof_end(ctx, ph);
    return GPLHR_OK;
  }
  if (use32)
    gplhr::combine_kernel<float><<<grid, gplhr::COMB_THREADS, smem, ctx->stream>>>(ctx->n, rows_per_cta, a);
  else
    gplhr::combine_kernel<double><<<grid, gplhr::COMB_THREADS, smem, ctx->stream>>>(ctx->n, rows_per_cta, a);
  CK(cudaGetLastError());
  if (c_store < c) {
    const int nc = c - c_store;
    gplhr::norm_reduce_kernel<<<(nc + 3) / 4, 128, 0, ctx->stream>>>(grid, nc, ctx->norm_part, ctx->d_norms);
    CK(cudaGetLastError());
  }
  prof_end(ctx, ph);
  return GPLHR_OK;
}

gplhr_status precond_apply_impl(gplhr_ctx* ctx, Blk X, int w, Blk Y);

gplhr_status gmres_apply(gplhr_ctx* ctx, Blk X, int w, Blk Y);

// The basic preconditioner T0 (Jacobi, block-Jacobi, CSR or I).
gplhr_status precond_apply_t0(gplhr_ctx* ctx, Blk X, int w, Blk Y) {
  if (ctx->prec == GPLHR_PREC_CSR) return precond_apply_impl(ctx, X, w, Y);  // counted as SpMM
  const double n = ctx->n;
  double fl = 0.0, by = 32.0 * n * w;
  if (ctx->prec == GPLHR_PREC_JACOBI) {
    fl = 6.0 * n * w;
    by += 16.0 * n;
  } else if (ctx->prec == GPLHR_PREC_BLOCK_JACOBI) {
    fl = 8.0 * n * ctx->bs * w;
    by += 16.0 * ((n + ctx->bs - 1) / ctx->bs) * ctx->bs * ctx->bs;
  }
  const int ph = prof_begin(ctx, KC_PREC, fl, by, (ctx->prec == GPLHR_PREC_NONE && X.p == Y.p) ? 0 : 1);
  gplhr_status st = precond_apply_impl(ctx, X, w, Y);
  prof_end(ctx, ph);
  return st;
}

// Y = T X: T0, or the inner block GMRES around it.
gplhr_status precond_apply(gplhr_ctx* ctx, Blk X, int w, Blk Y) {
  if (w <= 0) return GPLHR_OK;
  ctx->n_prec += 1;
  if (ctx->k1 > 0) {  // deflated T: (I - V1 V1^*) T (I - Q1 Q1^*), X projected in place
    TRY(project_out(ctx, Blk{ctx->hasB ? ctx->dQ1 : ctx->dV1, ctx->k1}, ctx->k1, X, w));
    TRY(precond_apply_t0(ctx, X, w, Y));
    return project_out(ctx, Blk{ctx->dV1, ctx->k1}, ctx->k1, Y, w);
  }
  return ctx->gm_steps > 0 ? gmres_apply(ctx, X, w, Y) : precond_apply_t0(ctx, X, w, Y);
}

gplhr_status precond_apply_impl(gplhr_ctx* ctx, Blk X, int w, Blk Y) {
  const int n = ctx->n;
  switch (ctx->prec) {
    case GPLHR_PREC_NONE: {
      if (X.p != Y.p) {
        launch_copy_block(ctx, grid_for((size_t)n * w, 256, 8 * ctx->num_sms), n, w, X.p, X.ld, Y.p, Y.ld);
        CK(cudaGetLastError());
      }
      return GPLHR_OK;
    }
    case GPLHR_PREC_JACOBI: {
      const int g = grid_for((size_t)n * w, 256, 8 * ctx->num_sms);
      if (ctx->rec)
        pk_rec(ctx, ctx->bulk32 ? gplhr::PK_JACOBI_F : gplhr::PK_JACOBI_D, g, 1, 0,
               gplhr::PkJacobi{n, w, X.ld, Y.ld, ctx->prec_data, X.p, Y.p});
      else if (ctx->bulk32)
        gplhr::jacobi_kernel<float><<<g, 256, 0, ctx->stream>>>(n, w, ctx->prec_data, X.p, X.ld, Y.p, Y.ld);
      else
        gplhr::jacobi_kernel<double><<<g, 256, 0, ctx->stream>>>(n, w, ctx->prec_data, X.p, X.ld, Y.p, Y.ld);
      CK(cudaGetLastError());
      return GPLHR_OK;
    }
    case GPLHR_PREC_BLOCK_JACOBI: {
      const int bs = ctx->bs;
      const int nblocks = (n + bs - 1) / bs;
      const int bpc = std::max(1, 1024 / (bs * w));
      const int grid = (nblocks + bpc - 1) / bpc;
      const size_t smem = (size_t)bpc * bs * w * sizeof(double2);
      if (ctx->rec) {
        const bool f32 = ctx->bulk32 && ctx->prec32;
        const gplhr::PkBj o{n, bs, w, X.ld, Y.ld, bpc, f32 ? (const void*)ctx->prec32 : (const void*)ctx->prec_data,
                            X.p, Y.p};
        pk_rec(ctx, f32 ? gplhr::PK_BJ_FF : ctx->bulk32 ? gplhr::PK_BJ_FD : gplhr::PK_BJ_DD, grid, 1, smem, o);
      } else if (ctx->bulk32 && ctx->prec32)
        gplhr::block_jacobi_kernel<float, float2><<<grid, gplhr::BJ_THREADS, smem, ctx->stream>>>(
            n, bs, w, ctx->prec32, X.p, X.ld, Y.p, Y.ld, bpc);
      else if (ctx->bulk32)
        gplhr::block_jacobi_kernel<float><<<grid, gplhr::BJ_THREADS, smem, ctx->stream>>>(
            n, bs, w, ctx->prec_data, X.p, X.ld, Y.p, Y.ld, bpc);
      else
        gplhr::block_jacobi_kernel<double><<<grid, gplhr::BJ_THREADS, smem, ctx->stream>>>(
            n, bs, w, ctx->prec_data, X.p, X.ld, Y.p, Y.ld, bpc);
      CK(cudaGetLastError());
      return GPLHR_OK;
    }
    case GPLHR_PREC_CSR: {
      if (X.p == Y.p) {  // out of place through a scratch block
        TRY(launch_spmm_one(ctx, ctx->Tcsr, nullptr, X, w, Blk{ctx->Tw1, ctx->k}, Blk{nullptr, 0}, ctx->bulk32));
        launch_copy_block(ctx, grid_for((size_t)n * w, 256, 8 * ctx->num_sms), n, w, ctx->Tw1, ctx->k, Y.p, Y.ld);
        CK(cudaGetLastError());
        return GPLHR_OK;
      }
      return launch_spmm_one(ctx, ctx->Tcsr, nullptr, X, w, Y, Blk{nullptr, 0}, ctx->bulk32);
    }
  }
  ctx->err = "unknown preconditioner";
  return GPLHR_EINVAL;
}

// X <- X - L (L^* X): one projection against the leading block L (wl columns).
gplhr_status project_out(gplhr_ctx* ctx, Blk L, int wl, Blk X, int w) {
  if (wl <= 0 || w <= 0) return GPLHR_OK;
  TRY(gram(ctx, L, wl, X, w, Blk{nullptr, 0}, 0, ctx->dProjC, nullptr, false, true, ctx->bulk32));
  return combine(ctx, {In{L, wl, ctx->dProjC, kMinusOne}}, X, w, true);
}

struct Extra {  // a block transformed alongside X (e.g. A P with P): E -= EL C; E <- E R^{-1}
  Blk E;
  Blk EL;
};

// orth of X against the leading block L (wl cols): block classical Gram-Schmidt
// twice interleaved with Cholesky QR twice,
//     pass: X -= L (L^* X);  G = X^* X = R^* R;  X <- X R^{-1},
// with a shifted Cholesky in the first pass when G is not numerically positive
// definite, followed then by a third pass (shifted Cholesky QR3).  Extras follow X.
// track: keep each pass's projection coefficients C_p (wl x w) in dTrackC and Cholesky
// factor R_p (w x w) in dTrackR, so that X_0 = L (C_0 + C_1 R_0 [+ C_2 R_1 R_0])
// + X_final (R_1 R_0 [R_2 R_1 R_0]) can be rebuilt on the host.
gplhr_status orth_against(gplhr_ctx* ctx, Blk L, int wl, Blk X, int w, const std::vector<Extra>& ex = {},
                          bool track = false) {
  if (w <= 0) return GPLHR_OK;
  const int smax2 = ctx->s_max * ctx->s_max;
  for (int pass = 0; pass < 3; ++pass) {
    // the third pass runs only when the first Cholesky needed the shift (decided on the
    // device); its work is not counted in the algorithmic totals
    const int* skip = pass == 2 ? ctx->d_status + 0 : nullptr;
    const bool cnt = pass < 2;
    const Blk none{nullptr, 0};
    if (wl > 0) {
      TRY(gram(ctx, L, wl, X, w, none, 0, ctx->dProjC, skip, false, cnt, ctx->bulk32));
      if (track)
        TRY(copy_async(ctx, ctx->dTrackC + (size_t)pass * ctx->trk, ctx->dProjC, (size_t)wl * w * sizeof(double2),
                       cudaMemcpyDeviceToDevice));
      TRY(combine(ctx, {In{L, wl, ctx->dProjC, kMinusOne}}, X, w, true, skip, none, -1, -1, cnt));
      for (const Extra& e : ex)
        TRY(combine(ctx, {In{e.EL, wl, ctx->dProjC, kMinusOne}}, e.E, w, true, skip, none, -1, -1, cnt));
    }
    TRY(gram(ctx, X, w, X, w, none, 0, ctx->dGram, skip, true, cnt));
    double2* Rinv = ctx->dRinv + (size_t)pass * smax2;
    const size_t smem = (size_t)2 * w * w * sizeof(double2);
    const int ph = prof_begin(ctx, KC_CHOL, 8.0 * w * w * w / 2.0, 48.0 * w * w);
    double2* Rout = track ? ctx->dTrackR + (size_t)pass * smax2 : nullptr;
    if (ctx->rec) {
      const bool glob = smem > gplhr::PK_CHOL_SMEM_MAX && ctx->pk_work;
      pk_rec(ctx, gplhr::PK_CHOL, 1, 1, glob ? 0 : smem,
             gplhr::PkChol{w, (int64_t)ctx->n, ctx->dGram, Rinv, ctx->d_status + pass, skip, ctx->d_diag, Rout,
                           glob ? ctx->pk_work : nullptr});
    } else {
      gplhr::chol_inv_kernel<<<1, 256, smem, ctx->stream>>>(w, (int64_t)ctx->n, ctx->dGram, Rinv,
                                                            ctx->d_status + pass, skip, ctx->d_diag, Rout);
    }
    prof_end(ctx, ph);
    CK(cudaGetLastError());
    TRY(combine(ctx, {In{X, w, Rinv, kOne}}, X, w, false, skip, none, -1, -1, cnt, -1, true));
    for (const Extra& e : ex)
      TRY(combine(ctx, {In{e.E, w, Rinv, kOne}}, e.E, w, false, skip, none, -1, -1, cnt, -1, true));
  }
  return GPLHR_OK;
}

// Accumulated factors of one tracked orth_against call from its passes' coefficients C_p
// (wl x w) and Cholesky factors R_p (w x w): X_0 = L C + X_final R with
// C = C_0 + C_1 R_0 [+ C_2 R_1 R_0] and R = R_1 R_0 [R_2 R_1 R_0].
void accumulate_tracks(const double2* hC, size_t strideC, const double2* hR, size_t strideR, int passes, int wl,
                       int w, std::vector<cd>& C, std::vector<cd>& R) {
  auto c_of = [&](int p, int i, int j) { const double2 v = hC[p * strideC + (size_t)i * w + j]; return cd(v.x, v.y); };
  auto r_of = [&](int p, int i, int j) { const double2 v = hR[p * strideR + (size_t)i * w + j]; return cd(v.x, v.y); };
  C.assign((size_t)wl * w, cd(0.0, 0.0));
  R.assign((size_t)w * w, cd(0.0, 0.0));
  for (int i = 0; i < wl; ++i)
    for (int j = 0; j < w; ++j) C[(size_t)i * w + j] = c_of(0, i, j);
  for (int i = 0; i < w; ++i)
    for (int j = i; j < w; ++j) R[(size_t)i * w + j] = r_of(0, i, j);
  for (int p = 1; p < passes; ++p) {
    std::vector<cd> Cn((size_t)wl * w), Rn((size_t)w * w, cd(0.0, 0.0));
    for (int i = 0; i < wl; ++i)
      for (int j = 0; j < w; ++j) {
        cd acc = C[(size_t)i * w + j];
        for (int t = 0; t <= j; ++t) acc += c_of(p, i, t) * R[(size_t)t * w + j];
        Cn[(size_t)i * w + j] = acc;
      }
    for (int i = 0; i < w; ++i)
      for (int j = i; j < w; ++j) {
        cd acc = 0.0;
        for (int t = i; t <= j; ++t) acc += r_of(p, i, t) * R[(size_t)t * w + j];
        Rn[(size_t)i * w + j] = acc;
      }
    C.swap(Cn);
    R.swap(Rn);
  }
}

// T R by s steps of block GMRES on K W = R, K = A - sigma B, zero start, right-
// preconditioned by T0 (Sec. 4): block Arnoldi K T0 V_j = V_{j+1} H(:, j) with the
// orthogonalisation of the sparse products (block CGS2 + Cholesky QR, tracked), then
// Y = argmin ||E_1 B_0 - H Y||_F (R = V_1 B_0) on the host, and T R = T0 (V_s Y).
gplhr_status gmres_apply_impl(gplhr_ctx* ctx, Blk X, int w, Blk Y);

// In the mixed mode the inner solve runs in FP32 in every phase: T is a preconditioner,
// whose accuracy sets the outer convergence rate but not the accuracy reached (residuals,
// projections, pencil and refinement of the outer iteration keep their own precision).
gplhr_status gmres_apply(gplhr_ctx* ctx, Blk X, int w, Blk Y) {
  const bool saved = ctx->bulk32;
  if (ctx->mixed) ctx->bulk32 = true;
  const gplhr_status st = gmres_apply_impl(ctx, X, w, Y);
  ctx->bulk32 = saved;
  return st;
}

gplhr_status gmres_apply_impl(gplhr_ctx* ctx, Blk X, int w, Blk Y) {
  const int s = ctx->gm_steps, k = ctx->k, n = ctx->n;
  const int ldv = (s + 1) * k;
  const int smax2 = ctx->s_max * ctx->s_max;
  const size_t per = 3 * ctx->trk + 3 * (size_t)k * k;  // pinned doubles2 per step
  auto Vb = [&](int j) { return Blk{ctx->gmV + (size_t)j * w, ldv}; };
  auto stash = [&](int j, int wl) -> gplhr_status {
    double2* h = ctx->h_gm + (size_t)j * per;
    for (int p = 0; p < 3; ++p) {
      if (wl > 0)
        CK(cudaMemcpyAsync(h + p * ctx->trk, ctx->dTrackC + p * ctx->trk, (size_t)wl * w * sizeof(double2),
                           cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaMemcpyAsync(h + 3 * ctx->trk + (size_t)p * k * k, ctx->dTrackR + (size_t)p * smax2,
                         (size_t)w * w * sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream));
    }
    CK(cudaMemcpyAsync(ctx->h_gm_status + j, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    ctx->d2h_bytes += (int64_t)(3 * ((size_t)wl * w + (size_t)w * w)) * sizeof(double2) + sizeof(int);
    return GPLHR_OK;
  };
  gplhr::copy_block_kernel<<<grid_for((size_t)n * w, 256, 8 * ctx->num_sms), 256, 0, ctx->stream>>>(
      n, w, X.p, X.ld, Vb(0).p, ldv);
  CK(cudaGetLastError());
  TRY(orth_against(ctx, Blk{nullptr, 0}, 0, Vb(0), w, {}, true));
  TRY(stash(0, 0));
  const Blk t{ctx->gmT, k}, ax{ctx->gmAX, k}, bx{ctx->gmBX, k};
  const double2 msig = make_double2(-ctx->sigma.real(), -ctx->sigma.imag());
  for (int j = 1; j <= s; ++j) {
    TRY(precond_apply_t0(ctx, Vb(j - 1), w, t));
    TRY(spmm_AB(ctx, t, w, ax, bx));
    const Blk b = ctx->hasB ? bx : t;
    const int ph = prof_begin(ctx, KC_OTHER, 8.0 * n * w, 48.0 * n * w);
    gplhr::axpby_kernel<<<grid_for((size_t)n * w, 256, 8 * ctx->num_sms), 256, 0, ctx->stream>>>(
        n, w, kOne, ax.p, ax.ld, msig, b.p, b.ld, Vb(j).p, ldv);
    prof_end(ctx, ph);
    CK(cudaGetLastError());
    TRY(orth_against(ctx, Blk{ctx->gmV, ldv}, j * w, Vb(j), w, {}, true));
    TRY(stash(j, j * w));
  }
  ctx->n_inner += s;
  CK(cudaStreamSynchronize(ctx->stream));
  // H ((s + 1) w x s w), block column j - 1 = [C_j; R_j] of step j; E = [B_0; 0]
  const int M = (s + 1) * w, N = s * w;
  std::vector<cd> H((size_t)M * N, cd(0.0, 0.0)), E((size_t)M * w, cd(0.0, 0.0)), C, R, Ys;
  for (int j = 0; j <= s; ++j) {
    const double2* h = ctx->h_gm + (size_t)j * per;
    const int passes = ctx->h_gm_status[j] != 0 ? 3 : 2;
    const int wl = j * w;
    accumulate_tracks(h, ctx->trk, h + 3 * ctx->trk, (size_t)k * k, passes, wl, w, C, R);
    for (int a = 0; a < w * w; ++a)
      if (!std::isfinite(R[a].real()) || !std::isfinite(R[a].imag())) {
        ctx->err = "non-finite Krylov basis in the inner GMRES";
        return GPLHR_ENUMERIC;
      }
    if (j == 0) {
      for (int i = 0; i < w; ++i)
        for (int c = 0; c < w; ++c) E[(size_t)i * w + c] = R[(size_t)i * w + c];
      continue;
    }
    const int col0 = (j - 1) * w;
    for (int i = 0; i < wl; ++i)
      for (int c = 0; c < w; ++c) H[(size_t)i * N + col0 + c] = C[(size_t)i * w + c];
    for (int i = 0; i < w; ++i)
      for (int c = 0; c < w; ++c) H[(size_t)(wl + i) * N + col0 + c] = R[(size_t)i * w + c];
  }
  gplhr::least_squares(H, M, N, E, w, Ys);
  for (int i = 0; i < N * w; ++i) ctx->h_gmY[i] = make_double2(Ys[i].real(), Ys[i].imag());
  CK(cudaMemcpyAsync(ctx->gmY, ctx->h_gmY, (size_t)N * w * sizeof(double2), cudaMemcpyHostToDevice, ctx->stream));
  ctx->h2d_bytes += (int64_t)N * w * sizeof(double2);
  TRY(combine(ctx, {In{Blk{ctx->gmV, ldv}, N, ctx->gmY, kOne}}, t, w, false));
  return precond_apply_t0(ctx, t, w, Y);
}

gplhr_status upload(gplhr_ctx* ctx, double2* dst, const double2* src, size_t elems) {
  ctx->h2d_bytes += (int64_t)(elems * sizeof(double2));
  return copy_async(ctx, dst, src, elems * sizeof(double2), cudaMemcpyHostToDevice);
}

// Pack a host matrix M (rows x cols of a SqMat, starting at (r0, c0)) into dst (row-major).
void pack(double2* dst, const SqMat& M, int r0, int rows, int c0, int cols) {
  for (int i = 0; i < rows; ++i)
    for (int j = 0; j < cols; ++j) dst[(size_t)i * cols + j] = d2(M(r0 + i, c0 + j));
}

Blk blkZ(gplhr_ctx* c, int col) { return Blk{c->Z + col, c->s_max}; }
Blk blkAZ(gplhr_ctx* c, int col) { return Blk{c->AZ + col, c->s_max}; }
Blk blkBZ(gplhr_ctx* c, int col) { return Blk{(c->hasB ? c->BZ : c->Z) + col, c->s_max}; }
Blk blkU(gplhr_ctx* c, int col) { return Blk{c->U + col, c->s_max}; }

// Residual R = AV M_B - BV M_A (all k columns, into Rw) and the backward errors of
// the pairs with x_j = V z_j (Sec. 5.1); host receives resid[].
// In parts: resid_issue stages the coefficients and issues (or records) the device
// segment, resid_post reads the norms once it completed.
gplhr_status resid_issue(gplhr_ctx* ctx, SqMat& Ze) {
  const int k = ctx->k;
  Ze = gplhr::tri_eigvecs(ctx->RA, ctx->RB);
  double2* h1 = ctx->h_small;
  double2* h2 = ctx->h_small + 2 * k * k;
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) {
      h1[i * 2 * k + j] = d2(ctx->MB(i, j));
      h2[i * 2 * k + j] = d2(ctx->MA(i, j));
      h1[i * 2 * k + k + j] = d2(Ze(i, j) * ctx->RB(j, j));
      h2[i * 2 * k + k + j] = d2(Ze(i, j) * ctx->RA(j, j));
    }
  TRY(run_segment(ctx, seg_key(3, 0, 0, 0, 0, ctx->bulk32 ? 1 : 0), [&]() -> gplhr_status {
    TRY(upload(ctx, ctx->dC1, h1, 2 * k * k));
    TRY(upload(ctx, ctx->dC2, h2, 2 * k * k));
    TRY(combine(ctx, {In{blkAZ(ctx, 0), k, ctx->dC1, kOne}, In{blkBZ(ctx, 0), k, ctx->dC2, kMinusOne}},
                Blk{ctx->Rw, k}, 2 * k, false, nullptr, Blk{nullptr, 0}, k, k));
    ctx->d2h_bytes += k * sizeof(double) + 3 * sizeof(int);
    TRY(copy_async(ctx, ctx->h_norms, ctx->d_norms, k * sizeof(double), cudaMemcpyDeviceToHost));
    TRY(copy_async(ctx, ctx->h_diag, ctx->d_diag, 3 * sizeof(int), cudaMemcpyDeviceToHost));
    return GPLHR_OK;
  }));
  return GPLHR_OK;
}

gplhr_status resid_post(gplhr_ctx* ctx, const SqMat& Ze) {
  const int k = ctx->k;
  ctx->resid.assign(k, 0.0);
  for (int j = 0; j < k; ++j) {
    double zn = 0.0;
    for (int i = 0; i <= j; ++i) zn += std::norm(Ze(i, j));
    const double a = std::abs(ctx->RA(j, j)), b = std::abs(ctx->RB(j, j));
    const double den = (b * ctx->normA + a * ctx->normB) * std::sqrt(zn);
    ctx->resid[j] = std::sqrt(ctx->h_norms[j]) / den;
    if (!std::isfinite(ctx->resid[j])) {
      ctx->err = "non-finite residual";
      return GPLHR_ENUMERIC;
    }
  }
  if (ctx->h_diag[1] != 0) {
    ctx->err = "orth(): Cholesky QR broke down even with the shifted first pass";
    return GPLHR_ESINGULAR;
  }
  if (ctx->h_diag[2] != 0) {
    ctx->err = "tensor-core product: wait for completion gave up";
    return GPLHR_ETIMEOUT;
  }
  return GPLHR_OK;
}

gplhr_status residuals(gplhr_ctx* ctx) {
  SqMat Ze;
  TRY(resid_issue(ctx, Ze));
  CK(cudaStreamSynchronize(ctx->stream));
  return resid_post(ctx, Ze);
}

// Host: sorted QZ of the s x s pencil in h_phipsi, returns Ybar_R, Ybar_L, Rbar_A, Rbar_B.
gplhr_status host_qz(gplhr_ctx* ctx, int s, SqMat& RAb, SqMat& RBb, SqMat& YLb, SqMat& YRb, int nsort = -1,
                     int nyl = -1, int nyr = -1) {
  SqMat Phi(s), Psi(s);
  for (int i = 0; i < s; ++i)
    for (int j = 0; j < s; ++j) {
      const double2 a = ctx->h_phipsi[(size_t)i * 2 * s + j];
      const double2 b = ctx->h_phipsi[(size_t)i * 2 * s + s + j];
      Phi(i, j) = cd(a.x, a.y);
      Psi(i, j) = cd(b.x, b.y);
      if (!std::isfinite(a.x) || !std::isfinite(a.y) || !std::isfinite(b.x) || !std::isfinite(b.y)) {
        ctx->err = "non-finite projected pencil";
        return GPLHR_ENUMERIC;
      }
    }
  ctx->n_qz += 1;
  if (!gplhr::ordered_qz(Phi, Psi, ctx->sigma, RAb, RBb, YLb, YRb, nsort, nyl, nyr)) {
    ctx->err = "QZ iteration did not converge";
    return GPLHR_ENUMERIC;
  }
  return GPLHR_OK;
}

void set_factors(gplhr_ctx* ctx, const SqMat& RAb, const SqMat& RBb) {
  const int k = ctx->k;
  ctx->RA = SqMat(k);
  ctx->RB = SqMat(k);
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) {
      ctx->RA(i, j) = RAb(i, j);
      ctx->RB(i, j) = RBb(i, j);
    }
  gplhr::m_factors(ctx->RA, ctx->RB, ctx->MA, ctx->MB);
}

gplhr_status start_steps(gplhr_ctx* ctx);

// Steps 1-4 of Algorithm 2.  Z[:, 0:k] must hold V0.
gplhr_status eig_start(gplhr_ctx* ctx);

gplhr_status start(gplhr_ctx* ctx) {
  if (ctx->eig) return eig_start(ctx);
  ctx->it = 0;
  ctx->q = 0;
  ctx->m = ctx->m0;
  ctx->hasP = false;
  ctx->n_spmm = ctx->n_prec = ctx->n_qz = ctx->n_inner = 0;
  ctx->h2d_bytes = ctx->d2h_bytes = 0;
  ctx->bulk32 = ctx->mixed;
  ctx->fp32_iters = 0;
  ctx->best_res = 1e300;
  ctx->since_best = 0;
  CK(cudaMemsetAsync(ctx->d_diag, 0, 3 * sizeof(int), ctx->stream));
  return start_steps(ctx);
}

// Steps 1-4 on the block in Z[:, 0:k]: V = orth(V), Q = orth((A - sigma B) V), ordered
// QZ of (Q^*AV, Q^*BV), V <- V YR, Q <- Q YL, M_A, M_B; then the residuals.
gplhr_status start_steps(gplhr_ctx* ctx) {
  const int k = ctx->k;
  if (ctx->k1 > 0) TRY(project_out(ctx, Blk{ctx->dV1, ctx->k1}, ctx->k1, blkZ(ctx, 0), k));  // deflation
  TRY(orth_against(ctx, Blk{nullptr, 0}, 0, blkZ(ctx, 0), k));                // V = orth(V0)
  TRY(spmm_AB(ctx, blkZ(ctx, 0), k, blkAZ(ctx, 0), blkBZ(ctx, 0)));        // AV, BV
  const double2 ms = d2(-ctx->sigma);
  const int ph = prof_begin(ctx, KC_OTHER, 8.0 * ctx->n * k, 48.0 * ctx->n * k);
  gplhr::axpby_kernel<<<grid_for((size_t)ctx->n * k, 256, 8 * ctx->num_sms), 256, 0, ctx->stream>>>(
      ctx->n, k, kOne, ctx->AZ, ctx->s_max, ms, blkBZ(ctx, 0).p, ctx->s_max, ctx->U, ctx->s_max);
  prof_end(ctx, ph);
  CK(cudaGetLastError());
  TRY(orth_against(ctx, Blk{nullptr, 0}, 0, blkU(ctx, 0), k));                // Q = orth((A - sigma B) V)
  TRY(gram(ctx, blkU(ctx, 0), k, blkAZ(ctx, 0), k, blkBZ(ctx, 0), k, ctx->dPhiPsi));
  ctx->d2h_bytes += (int64_t)2 * k * k * sizeof(double2);
  CK(cudaMemcpyAsync(ctx->h_phipsi, ctx->dPhiPsi, (size_t)2 * k * k * sizeof(double2), cudaMemcpyDeviceToHost,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  SqMat RAb, RBb, YLb, YRb;
  TRY(host_qz(ctx, k, RAb, RBb, YLb, YRb));
  double2* hy = ctx->h_small + 6 * k * k;  // residuals() reuses the first 4 k^2 entries
  double2* hl = hy + k * k;
  pack(hy, YRb, 0, k, 0, k);
  pack(hl, YLb, 0, k, 0, k);
  TRY(upload(ctx, ctx->dYR, hy, k * k));
  TRY(upload(ctx, ctx->dYL, hl, k * k));
  // V <- V YR, AV <- AV YR, BV <- BV YR, Q <- Q YL (in place)
  TRY(combine(ctx, {In{blkZ(ctx, 0), k, ctx->dYR, kOne}}, blkZ(ctx, 0), k, false));
  if (ctx->recompute) {
    TRY(spmm_AB(ctx, blkZ(ctx, 0), k, blkAZ(ctx, 0), blkBZ(ctx, 0)));
  } else {
    TRY(combine(ctx, {In{blkAZ(ctx, 0), k, ctx->dYR, kOne}}, blkAZ(ctx, 0), k, false));
    if (ctx->hasB) TRY(combine(ctx, {In{blkBZ(ctx, 0), k, ctx->dYR, kOne}}, blkBZ(ctx, 0), k, false));
  }
  TRY(combine(ctx, {In{blkU(ctx, 0), k, ctx->dYL, kOne}}, blkU(ctx, 0), k, false));
  set_factors(ctx, RAb, RBb);
  ctx->started = true;
  return residuals(ctx);
}

// Mixed mode: leave the FP32 bulk phase once the largest residual is below switch_tol,
// or, within two decades of switch_tol, has not dropped by 10 % over stall_iters
// iterations (the paper does not treat mixed precision; this switch rule is the
// library's, with the stall test restricted to where FP32 could be the floor).  The
// products AV, BV (and AP, BP when they are kept as combinations) are then formed again
// in FP64, and the residuals recomputed in FP64.
gplhr_status phase_update(gplhr_ctx* ctx) {
  if (!ctx->bulk32) return GPLHR_OK;
  double mx = 0.0;
  for (double r : ctx->resid) mx = std::max(mx, r);
  bool go = mx < ctx->switch_tol;
  if (mx < 0.9 * ctx->best_res) {
    ctx->best_res = mx;
    ctx->since_best = 0;
  } else if (mx < 100.0 * ctx->switch_tol && ++ctx->since_best >= ctx->stall_iters && ctx->stall_iters > 0) {
    // a plateau within two decades of switch_tol may be the FP32 floor; higher up it is
    // the method's own (irregular) convergence and the bulk phase continues
    go = true;
  }
  if (!go) return GPLHR_OK;
  ctx->bulk32 = false;
  const int k = ctx->k;
  if (!ctx->recompute && ctx->hasP)
    TRY(spmm_AB(ctx, Blk{ctx->Pb, k}, k, Blk{ctx->APb, k}, Blk{ctx->hasB ? ctx->BPb : ctx->Pb, k}));
  // Steps 1-4 again, in FP64, from the current V: V and Q orthonormal to FP64 accuracy
  // (the bulk phase leaves them orthonormal to FP32 accuracy only, and later iterations
  // only rotate Q by unitary factors), AV, BV and the Schur factors consistent with them.
  // P is kept.
  return start_steps(ctx);
}

// Convergence bookkeeping after residuals(): soft locking in order and m-adaptation
// (Sec. 3.6).  Locked pairs count as converged and stay locked; pair j can be locked
// only once pairs 0..j-1 are, so q grows by the run of pairs q, q+1, ... that meet tol,
// and m becomes the largest integer with m (k - q) <= m0 k (at most 20).  The solve has
// converged when every pair is locked (without locking: when every pair meets tol).
// Nothing converges or locks during the FP32 bulk phase.
int lock_lead(const gplhr_ctx* ctx) {
  int lead = ctx->lock ? ctx->q : 0;
  while (lead < ctx->k && lead < (int)ctx->resid.size() && ctx->resid[lead] <= ctx->tol) ++lead;
  return lead;
}

bool converged_update(gplhr_ctx* ctx) {
  const int k = ctx->k;
  if (ctx->bulk32) return false;
  const int lead = lock_lead(ctx);
  if (lead == k) {
    if (ctx->lock) ctx->q = k;
    return true;
  }
  if (ctx->lock && lead > ctx->q) {
    ctx->q = lead;
    ctx->m = std::min(ctx->m0 * k / (k - ctx->q), 20);
  }
  return false;
}

// Projected pencil without a second Gram (step 24).  U = [Q Qhat] was built so that
//   (A - sigma B) V       = Q (R_A - sigma R_B)                  (Prop. 3.2), and
//   (A - sigma B) [W S P] = Q C + Qhat R,  C = C_0 + C_1 R_0 (+ C_2 R_1 R_0),
//                                          R = R_1 R_0 (R_2 R_1 R_0)
// from the passes of its orthonormalisation, so F = U^*(A - sigma B) Z is the block upper
// triangular [[R_A - sigma R_B, C], [0, R]] and only Psi = U^* B Z needs a Gram product.
// The QZ runs on (F, Psi), whose eigenvalues are lambda - sigma (sorted by modulus), and
// Rbar_A = Rbar_F + sigma Rbar_Psi.
// Device part: Psi = U^* B Z and the tracked factors of U's construction, copied to the
// pinned host buffers (the caller synchronises before factored_pencil_qz).
gplhr_status factored_pencil_issue(gplhr_ctx* ctx, int s, int sk) {
  const int k = ctx->k;
  const int smax2 = ctx->s_max * ctx->s_max;
  TRY(gram(ctx, blkU(ctx, 0), s, blkBZ(ctx, 0), s, Blk{nullptr, 0}, 0, ctx->dPhiPsi));
  const size_t nC = (size_t)k * sk, nR = (size_t)sk * sk;
  double2* hC = ctx->h_track;                // 3 x nC
  double2* hR = ctx->h_track + 3 * nC;       // 3 x nR
  TRY(copy_async(ctx, ctx->h_phipsi, ctx->dPhiPsi, (size_t)s * s * sizeof(double2), cudaMemcpyDeviceToHost));
  for (int p = 0; p < 3; ++p) {
    TRY(copy_async(ctx, hC + p * nC, ctx->dTrackC + (size_t)p * ctx->trk, nC * sizeof(double2),
                   cudaMemcpyDeviceToHost));
    TRY(copy_async(ctx, hR + p * nR, ctx->dTrackR + (size_t)p * smax2, nR * sizeof(double2), cudaMemcpyDeviceToHost));
  }
  TRY(copy_async(ctx, ctx->h_status, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  ctx->d2h_bytes += (int64_t)((size_t)s * s + 3 * (nC + nR)) * sizeof(double2) + sizeof(int);
  return GPLHR_OK;
}

// Host part (after the synchronisation): the pencil (F, Psi) and its sorted QZ.
gplhr_status factored_pencil_qz(gplhr_ctx* ctx, int s, int sk, SqMat& RAb, SqMat& RBb, SqMat& YLb, SqMat& YRb,
                                int cv) {
  const int k = ctx->k;
  const size_t nC = (size_t)k * sk, nR = (size_t)sk * sk;
  double2* hPsi = ctx->h_phipsi;
  double2* hC = ctx->h_track;
  double2* hR = ctx->h_track + 3 * nC;
  const int passes = ctx->h_status[0] != 0 ? 3 : 2;
  auto Cm = [&](int p) {
    SqMat M(std::max(k, sk));
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < sk; ++j) M(i, j) = cd(hC[p * nC + i * sk + j].x, hC[p * nC + i * sk + j].y);
    return M;
  };
  auto Rm = [&](int p) {
    SqMat M(sk);
    for (int i = 0; i < sk; ++i)
      for (int j = 0; j < sk; ++j) M(i, j) = cd(hR[p * nR + i * sk + j].x, hR[p * nR + i * sk + j].y);
    return M;
  };
  // C and R accumulated over the passes: X_0 = Q C + Qhat R
  SqMat Cacc = Cm(0), Racc = Rm(0);
  for (int p = 1; p < passes; ++p) {
    SqMat Cp = Cm(p), Rp = Rm(p), Cn(std::max(k, sk)), Rn(sk);
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < sk; ++j) {
        cd acc = Cacc(i, j);
        for (int t = 0; t <= j; ++t) acc += Cp(i, t) * Racc(t, j);
        Cn(i, j) = acc;
      }
    for (int i = 0; i < sk; ++i)
      for (int j = i; j < sk; ++j) {
        cd acc = 0.0;
        for (int t = i; t <= j; ++t) acc += Rp(i, t) * Racc(t, j);
        Rn(i, j) = acc;
      }
    Cacc = Cn;
    Racc = Rn;
  }
  SqMat F(s), Psi(s);
  for (int i = 0; i < s; ++i)
    for (int j = 0; j < s; ++j) {
      const double2 b = hPsi[(size_t)i * s + j];
      Psi(i, j) = cd(b.x, b.y);
      if (!std::isfinite(b.x) || !std::isfinite(b.y)) {
        ctx->err = "non-finite projected pencil";
        return GPLHR_ENUMERIC;
      }
    }
  for (int i = 0; i < k; ++i) {
    for (int j = i; j < k; ++j) F(i, j) = ctx->RA(i, j) - ctx->sigma * ctx->RB(i, j);
    for (int j = 0; j < sk; ++j) F(i, k + j) = Cacc(i, j);
  }
  for (int i = 0; i < sk; ++i)
    for (int j = i; j < sk; ++j) F(k + i, k + j) = Racc(i, j);
  ctx->n_qz += 1;
  SqMat RFb;
  if (!gplhr::ordered_qz(F, Psi, cd(0.0, 0.0), RFb, RBb, YLb, YRb, cv, k, cv)) {
    ctx->err = "QZ iteration did not converge";
    return GPLHR_ENUMERIC;
  }
  RAb = SqMat(s);
  for (int i = 0; i < s; ++i)
    for (int j = i; j < s; ++j) RAb(i, j) = RFb(i, j) + ctx->sigma * RBb(i, j);
  return GPLHR_OK;
}

// One pass of the while loop of Algorithm 2 (steps 6-30), in parts: the plan (sizes of
// this iteration and the host staging of segment A), segment A (steps 7-24 up to the
// copies of the projected pencil to the host), the sorted QZ on the host, segment B
// (steps 25-28), and the host update of the factors (steps 29-30).  iterate_once runs
// them in order on the context's stream; the persistent batched iteration runs the
// device segments of many contexts in one kernel each.  Rw holds the residual.
struct IterPlan {
  int k, q, kk, m, sm, pslot, sP, s, sk, cv, flags, poff;
  bool withP, lob;
  SqMat RAb, RBb, YLb, YRb;
};

void iter_plan(gplhr_ctx* ctx, IterPlan& p) {
  p.k = ctx->k;
  p.q = ctx->q;
  p.kk = p.k - p.q;
  p.m = ctx->m;
  p.sm = ctx->s_max;
  p.withP = ctx->hasP && p.kk > 0 && ctx->p_mode != 2;
  p.lob = ctx->p_mode == 1;
  p.poff = p.lob ? p.q : 0;  // a LOBPCG-style P keeps its columns at V's positions
  p.pslot = p.k + (p.m + 1) * p.kk;
  p.sP = p.withP ? p.kk : 0;
  p.s = p.pslot + p.sP;
  p.sk = p.s - p.k;
  // only the leading k + kk positions of the ordering are used (V and a thick P)
  p.cv = ctx->p_mode == 0 ? p.k + p.kk : p.k;
  p.flags = (ctx->bulk32 ? 1 : 0) | (ctx->recompute ? 2 : 0) | (ctx->factored ? 4 : 0) | (p.withP ? 8 : 0) |
            (ctx->p_mode << 4) | (ctx->right_proj ? 0 : 64);
  // host staging of segment A: M_B, M_A of the active pairs for the S-recurrence
  if (p.m > 0) {
    double2* hm = ctx->h_small + 4 * p.k * p.k;
    for (int i = 0; i < p.kk; ++i)
      for (int j = 0; j < p.kk; ++j) {
        hm[i * p.kk + j] = d2(ctx->MB(p.q + i, p.q + j));
        hm[p.kk * p.kk + i * p.kk + j] = d2(ctx->MA(p.q + i, p.q + j));
      }
  }
}

// Segment A: steps 7-24 up to the copies of the projected pencil to the host.
gplhr_status iter_seg_a(gplhr_ctx* ctx, const IterPlan& p) {
  const int k = p.k, q = p.q, kk = p.kk, m = p.m, sm = p.sm, pslot = p.pslot, s = p.s, sk = p.sk;
  const Blk V = blkZ(ctx, 0), Q = blkU(ctx, 0);
  const Blk right = ctx->hasB ? Q : V;  // projector before T: (I - QQ^*), or (I - VV^*) if B = I
  return run_segment(ctx, seg_key(1, q, m, kk, s, p.flags), [&]() -> gplhr_status {
    // steps 7-8 / 10: W = (I - VV^*) T (I - QQ^*) R, active columns q..k-1
    Blk Ra{ctx->Rw + q, k};
    if (ctx->right_proj) TRY(project_out(ctx, right, k, Ra, kk));
    TRY(precond_apply(ctx, Ra, kk, blkZ(ctx, k)));
    TRY(orth_against(ctx, V, k, blkZ(ctx, k), kk));  // step 12 (with (I - VV^*))
    TRY(spmm_AB(ctx, blkZ(ctx, k), kk, blkAZ(ctx, k), blkBZ(ctx, k)));
    // steps 13-20: Krylov-Arnoldi blocks S_l
    if (m > 0) TRY(upload(ctx, ctx->dMBa, ctx->h_small + 4 * k * k, 2 * kk * kk));
    for (int l = 1; l <= m; ++l) {
      const int prev = k + (l - 1) * kk, cur = k + l * kk;
      Blk X{ctx->Rw, k};
      TRY(combine(ctx, {In{blkAZ(ctx, prev), kk, ctx->dMBa, kOne},
                        In{blkBZ(ctx, prev), kk, ctx->dMBa + kk * kk, kMinusOne}},
                  X, kk, false));
      if (ctx->right_proj) TRY(project_out(ctx, right, k, X, kk));
      TRY(precond_apply(ctx, X, kk, blkZ(ctx, cur)));
      TRY(orth_against(ctx, V, cur, blkZ(ctx, cur), kk));  // against V, W, S_1..S_{l-1}
      TRY(spmm_AB(ctx, blkZ(ctx, cur), kk, blkAZ(ctx, cur), blkBZ(ctx, cur)));
    }
    // step 21: P against V, W, S and orth; AP, BP follow by the same transforms
    if (p.withP) {
      const size_t nw = (size_t)ctx->n;
      const int ncopy = ctx->recompute ? 1 : (ctx->hasB ? 3 : 2);
      const int gcp = grid_for(nw * kk, 256, 8 * ctx->num_sms);
      const int ph = prof_begin(ctx, KC_OTHER, 0.0, 32.0 * ctx->n * kk * ncopy, ncopy);
      launch_copy_block(ctx, gcp, ctx->n, kk, ctx->Pb + p.poff, k, ctx->Z + pslot, sm);
      if (!ctx->recompute) {
        launch_copy_block(ctx, gcp, ctx->n, kk, ctx->APb + p.poff, k, ctx->AZ + pslot, sm);
        if (ctx->hasB) launch_copy_block(ctx, gcp, ctx->n, kk, ctx->BPb + p.poff, k, ctx->BZ + pslot, sm);
      }
      prof_end(ctx, ph);
      CK(cudaGetLastError());
      if (ctx->recompute) {
        TRY(orth_against(ctx, V, pslot, blkZ(ctx, pslot), kk));
        TRY(spmm_AB(ctx, blkZ(ctx, pslot), kk, blkAZ(ctx, pslot), blkBZ(ctx, pslot)));
      } else {
        std::vector<Extra> ex{Extra{blkAZ(ctx, pslot), blkAZ(ctx, 0)}};
        if (ctx->hasB) ex.push_back(Extra{blkBZ(ctx, pslot), blkBZ(ctx, 0)});
        TRY(orth_against(ctx, V, pslot, blkZ(ctx, pslot), kk, ex));
      }
    }
    // steps 23-24: Qhat = orth((A - sigma B) [W S P]) against Q;  U = [Q Qhat]
    const int ph_ax = prof_begin(ctx, KC_OTHER, 8.0 * ctx->n * sk, 48.0 * ctx->n * sk);
    launch_axpby(ctx, grid_for((size_t)ctx->n * sk, 256, 8 * ctx->num_sms), ctx->n, sk, kOne, ctx->AZ + k, sm,
                 d2(-ctx->sigma), blkBZ(ctx, k).p, sm, ctx->U + k, sm);
    prof_end(ctx, ph_ax);
    CK(cudaGetLastError());
    TRY(orth_against(ctx, Q, k, blkU(ctx, k), sk, {}, ctx->factored));
    if (ctx->factored) return factored_pencil_issue(ctx, s, sk);
    // step 24: projected pencil (U^* A Z, U^* B Z) by two Gram products
    TRY(gram(ctx, blkU(ctx, 0), s, blkAZ(ctx, 0), s, blkBZ(ctx, 0), s, ctx->dPhiPsi));
    ctx->d2h_bytes += (int64_t)2 * s * s * sizeof(double2);
    return copy_async(ctx, ctx->h_phipsi, ctx->dPhiPsi, (size_t)2 * s * s * sizeof(double2), cudaMemcpyDeviceToHost);
  });
}

// Host, after segment A completed: the sorted QZ and the staging of segment B.
gplhr_status iter_qz(gplhr_ctx* ctx, IterPlan& p) {
  const int k = p.k, s = p.s, cv = p.cv;
  if (ctx->factored)
    TRY(factored_pencil_qz(ctx, s, p.sk, p.RAb, p.RBb, p.YLb, p.YRb, cv));
  else
    TRY(host_qz(ctx, s, p.RAb, p.RBb, p.YLb, p.YRb, cv, k, cv));
  // steps 25-28: V = Z Ybar_R(:, 1:k), P = Z Ybar_R(:, k+1:k+kk), Q = U Ybar_L(:, 1:k)
  double2* hy = ctx->h_small + 6 * k * k;
  double2* hl = hy + (size_t)s * cv;
  pack(hy, p.YRb, 0, s, 0, cv);
  pack(hl, p.YLb, 0, s, 0, k);
  return GPLHR_OK;
}

// Segment B: steps 25-28.
gplhr_status iter_seg_b(gplhr_ctx* ctx, const IterPlan& p) {
  const int k = p.k, s = p.s, cv = p.cv, sm = p.sm;
  const bool lob = p.lob;
  const double2* hy = ctx->h_small + 6 * k * k;
  const double2* hl = hy + (size_t)s * cv;
  return run_segment(ctx, seg_key(2, p.q, p.m, p.kk, s, p.flags), [&]() -> gplhr_status {
    TRY(upload(ctx, ctx->dYR, hy, (size_t)s * cv));
    TRY(upload(ctx, ctx->dYL, hl, (size_t)s * k));
    const int nb = (int)grid_for((size_t)ctx->n * k, 256, 8 * ctx->num_sms);
    if (lob) {  // V_old (and A V_old, B V_old) into the P buffers before the update
      const int ph = prof_begin(ctx, KC_OTHER, 0.0, 32.0 * ctx->n * k, 1);
      launch_copy_block(ctx, nb, ctx->n, k, ctx->Z, sm, ctx->Pb, k);
      if (!ctx->recompute) {
        launch_copy_block(ctx, nb, ctx->n, k, ctx->AZ, sm, ctx->APb, k);
        if (ctx->hasB) launch_copy_block(ctx, nb, ctx->n, k, ctx->BZ, sm, ctx->BPb, k);
      }
      prof_end(ctx, ph);
      CK(cudaGetLastError());
    }
    TRY(combine(ctx, {In{blkZ(ctx, 0), s, ctx->dYR, kOne}}, blkZ(ctx, 0), cv, false, nullptr, Blk{ctx->Pb, k}, k));
    if (ctx->recompute) {
      // AV, BV by fresh sparse products (AP, BP are formed after P's orth next iteration)
      TRY(spmm_AB(ctx, blkZ(ctx, 0), k, blkAZ(ctx, 0), blkBZ(ctx, 0)));
    } else {
      TRY(combine(ctx, {In{blkAZ(ctx, 0), s, ctx->dYR, kOne}}, blkAZ(ctx, 0), cv, false, nullptr,
                  Blk{ctx->APb, k}, k));
      if (ctx->hasB)
        TRY(combine(ctx, {In{blkBZ(ctx, 0), s, ctx->dYR, kOne}}, blkBZ(ctx, 0), cv, false, nullptr,
                    Blk{ctx->BPb, k}, k));
    }
    TRY(combine(ctx, {In{blkU(ctx, 0), s, ctx->dYL, kOne}}, blkU(ctx, 0), k, false));
    if (lob) {  // Eq. P_lobpcg with C = I: P = V - V_old (A P, B P likewise)
      const int ph = prof_begin(ctx, KC_OTHER, 8.0 * ctx->n * k, 48.0 * ctx->n * k, 1);
      launch_axpby(ctx, nb, ctx->n, k, kOne, ctx->Z, sm, kMinusOne, ctx->Pb, k, ctx->Pb, k);
      if (!ctx->recompute) {
        launch_axpby(ctx, nb, ctx->n, k, kOne, ctx->AZ, sm, kMinusOne, ctx->APb, k, ctx->APb, k);
        if (ctx->hasB) launch_axpby(ctx, nb, ctx->n, k, kOne, ctx->BZ, sm, kMinusOne, ctx->BPb, k, ctx->BPb, k);
      }
      prof_end(ctx, ph);
      CK(cudaGetLastError());
    }
    return GPLHR_OK;
  });
}

// Host, after segment B was issued: steps 29-30.
void iter_finish(gplhr_ctx* ctx, const IterPlan& p) {
  ctx->hasP = ctx->p_mode != 2;
  set_factors(ctx, p.RAb, p.RBb);
  ctx->it += 1;
}

gplhr_status iterate_once(gplhr_ctx* ctx) {
  IterPlan p;
  iter_plan(ctx, p);
  TRY(iter_seg_a(ctx, p));
  CK(cudaStreamSynchronize(ctx->stream));
  TRY(iter_qz(ctx, p));
  TRY(iter_seg_b(ctx, p));
  iter_finish(ctx, p);
  return GPLHR_OK;
}

void fill_info(gplhr_ctx* ctx, gplhr_info* info) {
  if (!info) return;
  std::memset(info, 0, sizeof(*info));
  info->iters = ctx->it;
  info->nconv = ctx->bulk32 ? 0 : lock_lead(ctx);
  info->m = ctx->m;
  info->n_orth_fallback = ctx->h_diag ? ctx->h_diag[0] : 0;
  info->fp32_iters = ctx->fp32_iters;
  info->bulk = ctx->bulk32 ? 1 : 0;
  info->n_spmm = ctx->n_spmm;
  info->n_prec = ctx->n_prec;
  info->n_inner = ctx->n_inner;
  info->n_qz = ctx->n_qz;
  info->n_launch = ctx->n_launch;
  info->h2d_bytes = ctx->h2d_bytes;
  info->d2h_bytes = ctx->d2h_bytes;
  for (int j = 0; j < ctx->k && j < 64 && j < (int)ctx->resid.size(); ++j) info->resid[j] = ctx->resid[j];
}

gplhr_status eig_run(gplhr_ctx* ctx, int niter, gplhr_info* info, bool* conv_out);

gplhr_status run_iterations(gplhr_ctx* ctx, int niter, gplhr_info* info, bool* conv_out) {
  if (ctx->eig) return eig_run(ctx, niter, info, conv_out);
  TRY(phase_update(ctx));
  bool conv = converged_update(ctx);
  for (int i = 0; i < niter && !conv; ++i) {
    if (ctx->bulk32) ctx->fp32_iters += 1;
    TRY(iterate_once(ctx));
    TRY(residuals(ctx));
    TRY(phase_update(ctx));
    conv = converged_update(ctx);
  }
  fill_info(ctx, info);
  if (conv_out) *conv_out = conv;
  return GPLHR_OK;
}

// -------------------------------------------------- persistent batched iteration ----
// Many contexts (pencils of uneven size, or shifts over one pencil) iterate in lockstep,
// and each device segment of an iteration (A: steps 7-24, B: steps 25-28, C: the
// residual and its norms) runs for all of them in ONE launch of the persistent kernel of
// persist.cuh: the host records each context's launches (the same kernels, grids and
// arguments as gplhr_iterate, on DFMA, with grids sized to the context's share of the
// SMs), merges them into one queue, and the kernel runs each context's launches in order,
// the contexts independently.  An iteration of the whole batch is three launches and two
// host round trips (the
// pencils for the host QZ, the residual norms for locking), instead of ~100 launches
// per context.
struct PkBuf {
  unsigned char* host = nullptr;  // pinned staging of a program
  unsigned char* dev = nullptr;
  size_t cap = 0;
};

struct PkRunner {
  int dev = 0, num_sms = 0;
  cudaStream_t stream = nullptr;
  PkBuf buf[3];  // one per segment kind, so a program is not overwritten while its copy is pending
  gplhr::PkQueue* queue = nullptr;
  int* derr = nullptr;
  int* herr = nullptr;
  unsigned long long limit_ns = 0;
  int probe = 0;
  int64_t launches = 0, steps = 0, ops = 0;
  int grid = 0;
  // host time recording segments, merging and uploading programs, in the host QZ, and
  // waiting for the device (ms)
  double record_ms = 0.0, build_ms = 0.0, qz_ms = 0.0, wait_ms = 0.0;
  std::vector<double2*> work;  // per context: global work of its wide Cholesky factorisations
  // the last program of each segment kind: its recordings and device program
  std::vector<const PkRecorder*> last_recs[3];
  gplhr::PkProgram last_prog[3] = {};
  size_t last_smem[3] = {0, 0, 0}, last_nsteps[3] = {0, 0, 0}, last_nops[3] = {0, 0, 0};
  std::string err;
  ~PkRunner() {
    for (PkBuf& b : buf) {
      if (b.host) cudaFreeHost(b.host);
      if (b.dev) cudaFree(b.dev);
    }
    if (queue) cudaFree(queue);
    for (double2* w : work)
      if (w) cudaFree(w);
    if (derr) cudaFree(derr);
    if (herr) cudaFreeHost(herr);
    if (stream) cudaStreamDestroy(stream);
  }
};

constexpr double kPkShare = 4.0;

#define PKCK(call)                                                     \
  do {                                                                 \
    cudaError_t e_ = (call);                                           \
    if (e_ != cudaSuccess) {                                           \
      R.err = std::string(#call) + ": " + cudaGetErrorString(e_);      \
      return GPLHR_ECUDA;                                              \
    }                                                                  \
  } while (0)

// Merge the recorded segments into one program and run it on R.stream: host-to-device
// copies, the program's upload, the persistent kernel, device-to-host copies.
gplhr_status pk_launch_impl(PkRunner& R, int seg, const std::vector<const PkRecorder*>& recs);
gplhr_status pk_launch(PkRunner& R, int seg, const std::vector<const PkRecorder*>& recs) {
  const auto t0 = std::chrono::steady_clock::now();
  const gplhr_status st = pk_launch_impl(R, seg, recs);
  R.build_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return st;
}

// The persistent kernel on R.stream: its queue and finish counts zeroed, cooperative (all
// CTAs resident).
gplhr_status pk_run(PkRunner& R, gplhr::PkProgram prog, size_t smem, size_t nsteps, size_t nops) {
  if (smem > 48 * 1024)
    PKCK(cudaFuncSetAttribute(gplhr::persistent_segment_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem));
  int occ = 0;
  PKCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, gplhr::persistent_segment_kernel, gplhr::PK_THREADS,
                                                     smem));
  if (occ < 1) {
    R.err = "persistent kernel: no CTA fits an SM with " + std::to_string(smem) + " bytes of shared memory";
    return GPLHR_EINVAL;
  }
  R.grid = R.num_sms * std::min(occ, gplhr::PK_CTAS_PER_SM);
  PKCK(cudaMemsetAsync(R.queue, 0, sizeof(gplhr::PkQueue), R.stream));
  PKCK(cudaMemsetAsync(prog.claimed, 0, (size_t)(2 * prog.nops + prog.nctx) * sizeof(int), R.stream));
  void* kargs[] = {&prog, &R.queue, &R.derr, &R.limit_ns, &R.probe};
  PKCK(cudaLaunchCooperativeKernel((const void*)gplhr::persistent_segment_kernel, dim3(R.grid),
                                   dim3(gplhr::PK_THREADS), kargs, smem, R.stream));
  R.launches += 1;
  R.steps += (int64_t)nsteps;
  R.ops += (int64_t)nops;
  return GPLHR_OK;
}

gplhr_status pk_launch_impl(PkRunner& R, int seg, const std::vector<const PkRecorder*>& recs) {
  // the same recordings as the last launch of this segment kind: its program is on the
  // device already (recordings are immutable once made)
  if (!recs.empty() && recs == R.last_recs[seg])
    return pk_run(R, R.last_prog[seg], R.last_smem[seg], R.last_nsteps[seg], R.last_nops[seg]);
  R.last_recs[seg].clear();
  // each context's sequence: its host-to-device copies, its recorded launches, its
  // device-to-host copies (the copies run inside the kernel: the device reads and writes
  // the host's pinned staging directly); contexts in the given (priority) order
  size_t nops = 0, nsteps = 0, argbytes = 0, smem = 0;
  const size_t nctx = recs.size();
  const size_t rawsz = (sizeof(gplhr::PkRaw) + 15) & ~(size_t)15;
  for (const PkRecorder* r : recs) {
    const size_t len = r->pre.size() + r->ops.size() + r->post.size();
    nops += len;
    nsteps = std::max(nsteps, len);
    argbytes += (r->pre.size() + r->post.size()) * rawsz;
    for (const PkRecorder::Op& o : r->ops) {
      argbytes += (o.size + 15) & ~(size_t)15;
      smem = std::max(smem, o.smem);
    }
  }
  if (nops == 0) return GPLHR_OK;
  if (argbytes > 0xFFFFFFFFull || nops > (size_t)INT_MAX / 2) {
    R.err = "persistent program: too large";
    return GPLHR_EINVAL;
  }
  auto al = [](size_t x) { return (x + 15) & ~(size_t)15; };
  const size_t o_ops = 0, o_vc = al(o_ops + nops * sizeof(gplhr::PkOp)), o_cf = al(o_vc + nops * sizeof(int)),
               o_cn = al(o_cf + nctx * sizeof(int)), o_zero = al(o_cn + nctx * sizeof(int)),
               zbytes = (2 * nops + nctx) * sizeof(int), o_args = al(o_zero + zbytes), total = o_args + argbytes;
  PkBuf& B = R.buf[seg];
  if (B.cap < total) {
    if (B.host) cudaFreeHost(B.host);
    if (B.dev) cudaFree(B.dev);
    B.host = nullptr;
    B.dev = nullptr;
    B.cap = 0;
    const size_t cap = total + total / 2;
    if (cudaMallocHost(&B.host, cap) != cudaSuccess || cudaMalloc(&B.dev, cap) != cudaSuccess) {
      R.err = "persistent program: allocation failed";
      return GPLHR_ENOMEM;
    }
    B.cap = cap;
  }
  gplhr::PkOp* ops = reinterpret_cast<gplhr::PkOp*>(B.host + o_ops);
  int* vcount = reinterpret_cast<int*>(B.host + o_vc);
  int* ctx_first = reinterpret_cast<int*>(B.host + o_cf);
  int* ctx_nops = reinterpret_cast<int*>(B.host + o_cn);
  size_t no = 0, ao = 0;
  auto put = [&](int kind, int gx, int gy, const void* arg, size_t size) {
    std::memcpy(B.host + o_args + ao, arg, size);
    ops[no] = gplhr::PkOp{kind, gx, gy, (unsigned)ao};
    vcount[no] = gx * gy;
    ao += (size + 15) & ~(size_t)15;
    ++no;
  };
  auto put_copy = [&](const PkRecorder::Copy& c) {
    const gplhr::PkRaw a{(const unsigned char*)c.src, (unsigned char*)c.dst, (int64_t)c.bytes};
    put(gplhr::PK_COPY_RAW, (int)std::max<size_t>(1, std::min<size_t>(8, c.bytes / 4096)), 1, &a, sizeof(a));
  };
  for (size_t ci = 0; ci < nctx; ++ci) {
    const PkRecorder* r = recs[ci];
    ctx_first[ci] = (int)no;
    for (const PkRecorder::Copy& c : r->pre) put_copy(c);
    for (const PkRecorder::Op& o : r->ops) put(o.kind, o.gx, o.gy, r->args.data() + o.off, o.size);
    for (const PkRecorder::Copy& c : r->post) put_copy(c);
    ctx_nops[ci] = (int)no - ctx_first[ci];
  }
  PKCK(cudaMemcpyAsync(B.dev, B.host, o_zero, cudaMemcpyHostToDevice, R.stream));  // ops, counts, contexts
  PKCK(cudaMemcpyAsync(B.dev + o_args, B.host + o_args, argbytes, cudaMemcpyHostToDevice, R.stream));
  int* zero = reinterpret_cast<int*>(B.dev + o_zero);
  gplhr::PkProgram prog{reinterpret_cast<const gplhr::PkOp*>(B.dev + o_ops),
                        B.dev + o_args,
                        reinterpret_cast<const int*>(B.dev + o_vc),
                        reinterpret_cast<const int*>(B.dev + o_cf),
                        reinterpret_cast<const int*>(B.dev + o_cn),
                        zero,
                        zero + nops,
                        zero + 2 * nops,
                        (int)nops,
                        (int)nctx};
  TRY(pk_run(R, prog, smem, nsteps, nops));
  R.last_recs[seg] = recs;
  R.last_prog[seg] = prog;
  R.last_smem[seg] = smem;
  R.last_nsteps[seg] = nsteps;
  R.last_nops[seg] = nops;
  return GPLHR_OK;
}

// Wait for R.stream; GPLHR_ETIMEOUT if a wait of the kernel gave up.
gplhr_status pk_sync(PkRunner& R) {
  PKCK(cudaMemcpyAsync(R.herr, R.derr, sizeof(int), cudaMemcpyDeviceToHost, R.stream));
  const auto t0 = std::chrono::steady_clock::now();
  PKCK(cudaStreamSynchronize(R.stream));
  R.wait_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (*R.herr != 0) {
    R.err = "persistent kernel: no launch became ready within the wait limit";
    return GPLHR_ETIMEOUT;
  }
  return GPLHR_OK;
}

// A fixed pool of host threads for the per-context host work of the persistent batch
// (recording, QZ, residual bookkeeping): spawning threads for each of the five parallel
// phases of an iteration costs more than the work itself.
class PkPool {
 public:
  PkPool(int nthreads, int dev) : dev_(dev) {
    for (int t = 1; t < nthreads; ++t) th_.emplace_back([this]() { loop(); });
  }
  ~PkPool() {
    {
      std::lock_guard<std::mutex> g(m_);
      stop_ = true;
    }
    cv_.notify_all();
    for (auto& t : th_) t.join();
  }
  // f(idx[j]) for every j, on the pool and the calling thread; returns when all are done.
  void run(const std::vector<int>& idx, const std::function<void(int)>& f) {
    if (idx.empty()) return;
    {
      std::lock_guard<std::mutex> g(m_);
      idx_ = &idx;
      f_ = &f;
      next_ = 0;
      done_ = 0;
      ++gen_;
    }
    cv_.notify_all();
    work();
    std::unique_lock<std::mutex> g(m_);
    done_cv_.wait(g, [&]() { return done_ == (int)idx.size(); });
    idx_ = nullptr;
    f_ = nullptr;
  }

 private:
  void work() {
    for (;;) {
      int j;
      const std::vector<int>* idx;
      const std::function<void(int)>* f;
      {
        std::lock_guard<std::mutex> g(m_);
        if (!idx_ || next_ >= (int)idx_->size()) return;
        j = next_++;
        idx = idx_;
        f = f_;
      }
      (*f)((*idx)[j]);
      {
        std::lock_guard<std::mutex> g(m_);
        if (++done_ == (int)idx->size()) done_cv_.notify_all();
      }
    }
  }
  void loop() {
    cudaSetDevice(dev_);
    uint64_t seen = 0;
    for (;;) {
      {
        std::unique_lock<std::mutex> g(m_);
        cv_.wait(g, [&]() { return stop_ || gen_ != seen; });
        if (stop_) return;
        seen = gen_;
      }
      work();
    }
  }
  int dev_;
  std::vector<std::thread> th_;
  std::mutex m_;
  std::condition_variable cv_, done_cv_;
  const std::vector<int>* idx_ = nullptr;
  const std::function<void(int)>* f_ = nullptr;
  int next_ = 0, done_ = 0;
  uint64_t gen_ = 0;
  bool stop_ = false;
};

// The persistent batched iteration over started contexts: each runs until it converges,
// fails, or has run its budget (iters_cap[i] total iterations).
gplhr_status pk_iterate(int nctx, gplhr_ctx* const* ctxs, const std::vector<int>& iters_cap, int nthreads,
                        std::vector<gplhr_status>& st, std::vector<char>& conv, PkRunner& R) {
  st.assign(nctx, GPLHR_OK);
  conv.assign(nctx, 0);
  PKCK(cudaGetDevice(&R.dev));
  PKCK(cudaDeviceGetAttribute(&R.num_sms, cudaDevAttrMultiProcessorCount, R.dev));
  PKCK(cudaStreamCreateWithFlags(&R.stream, cudaStreamNonBlocking));
  PKCK(cudaMalloc(&R.queue, sizeof(gplhr::PkQueue)));
  PKCK(cudaMalloc(&R.derr, sizeof(int)));
  PKCK(cudaMemset(R.derr, 0, sizeof(int)));
  PKCK(cudaMallocHost(&R.herr, sizeof(int)));
  // the kernel's wait limit: the contexts' wait limit (tests of at most 20 us each)
  int tries = gplhr::TC_WAIT_TRIES;
  for (int i = 0; i < nctx; ++i) {
    tries = std::min(tries, ctxs[i]->tc_wait_tries);
    if (ctxs[i]->tc_probe) R.probe = 1;
  }
  R.limit_ns = (unsigned long long)tries * 20000ull;
  // DFMA kernels (the tensor-core pipelines keep their own CTA shape), grids sized to a
  // share of the SMs proportional to the context's rows: kPkShare x the SM count in all,
  // so that each step has a few virtual CTAs per persistent CTA (measured on the batched
  // workload, 80 contexts, 2 resident CTAs per SM: share 1 / 2 / 4 / 8 / 16 -> 33.3 / 30.5 /
  // 28.6 / 30.3 / 31.2 ms per FP64 batch iteration; with 4: 4 / 8 -> 20.6 / 22.0 ms)
  double nsum = 0.0;
  for (int i = 0; i < nctx; ++i) nsum += ctxs[i]->n;
  std::vector<int> saved_sms(nctx);
  std::vector<char> saved_tc(nctx);
  R.work.assign(nctx, nullptr);
  for (int i = 0; i < nctx; ++i)  // (before any context is changed: an early return leaves them as they were)
    if (gplhr::PK_CHOL_SMEM_MAX < (size_t)2 * ctxs[i]->s_max * ctxs[i]->s_max * sizeof(double2))
      PKCK(cudaMalloc(&R.work[i], (size_t)2 * ctxs[i]->s_max * ctxs[i]->s_max * sizeof(double2)));
  for (int i = 0; i < nctx; ++i) {
    gplhr_ctx* c = ctxs[i];
    c->pk_work = R.work[i];
    saved_sms[i] = c->num_sms;
    saved_tc[i] = c->tc;
    c->num_sms = std::max(1, (int)std::lround(kPkShare * R.num_sms * c->n / nsum));
    c->tc = false;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) st[i] = GPLHR_ECUDA;
  }
  std::vector<int> all(nctx);
  for (int i = 0; i < nctx; ++i) all[i] = i;
  PkPool pool(std::max(1, std::min(nthreads, nctx)), R.dev);
  pool.run(all, [&](int i) {
    if (st[i] != GPLHR_OK) return;
    st[i] = phase_update(ctxs[i]);
    if (st[i] == GPLHR_OK) conv[i] = converged_update(ctxs[i]);
  });
  std::vector<IterPlan> plan(nctx);
  std::vector<std::map<uint64_t, gplhr_ctx::PkCached>> cache(nctx);
  std::vector<SqMat> Ze(nctx);
  gplhr_status fatal = GPLHR_OK;
  // record the contexts' segments on host threads (each context records into its own
  // recorder), then keep the ones that succeeded, in context order
  auto record = [&](std::vector<int>& act, const std::function<gplhr_status(int)>& issue) {
    const auto t0 = std::chrono::steady_clock::now();
    pool.run(act, [&](int i) {
      ctxs[i]->pk_cache = &cache[i];
      ctxs[i]->rec_last = nullptr;
      st[i] = issue(i);
      ctxs[i]->pk_cache = nullptr;
      if (st[i] == GPLHR_OK && !ctxs[i]->rec_last) {
        ctxs[i]->err = "persistent batch: a segment recorded nothing";
        st[i] = GPLHR_EINVAL;
      }
    });
    std::vector<const PkRecorder*> rs;
    std::vector<int> keep;
    for (int i : act)
      if (st[i] == GPLHR_OK) {
        rs.push_back(ctxs[i]->rec_last);
        keep.push_back(i);
      }
    act.swap(keep);
    R.record_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return rs;
  };
  for (;;) {
    std::vector<int> act;
    for (int i = 0; i < nctx; ++i)
      if (st[i] == GPLHR_OK && !conv[i] && ctxs[i]->it < iters_cap[i]) act.push_back(i);
    if (act.empty()) break;
    // the persistent kernel serves contexts in this order when several are ready: the
    // largest first (their chains of launches are the longest)
    std::stable_sort(act.begin(), act.end(), [&](int x, int y) { return ctxs[x]->n > ctxs[y]->n; });
    for (int i : act) {
      if (ctxs[i]->bulk32) ctxs[i]->fp32_iters += 1;
      iter_plan(ctxs[i], plan[i]);
    }
    // segment A, then the host QZ of every pencil
    fatal = pk_launch(R, 0, record(act, [&](int i) { return iter_seg_a(ctxs[i], plan[i]); }));
    if (fatal == GPLHR_OK) fatal = pk_sync(R);
    if (fatal != GPLHR_OK) break;
    auto tq = std::chrono::steady_clock::now();
    pool.run(act, [&](int i) { st[i] = iter_qz(ctxs[i], plan[i]); });
    R.qz_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tq).count();
    std::vector<int> act_b;
    for (int i : act)
      if (st[i] == GPLHR_OK) act_b.push_back(i);
    // segment B, the factors, segment C
    fatal = pk_launch(R, 1, record(act_b, [&](int i) { return iter_seg_b(ctxs[i], plan[i]); }));
    if (fatal != GPLHR_OK) break;
    for (int i : act_b) iter_finish(ctxs[i], plan[i]);
    fatal = pk_launch(R, 2, record(act_b, [&](int i) { return resid_issue(ctxs[i], Ze[i]); }));
    if (fatal == GPLHR_OK) fatal = pk_sync(R);
    if (fatal != GPLHR_OK) break;
    // residuals, the precision switch (on the context's own stream) and locking
    pool.run(act_b, [&](int i) {
      gplhr_ctx* c = ctxs[i];
      st[i] = resid_post(c, Ze[i]);
      if (st[i] == GPLHR_OK) st[i] = phase_update(c);
      if (st[i] == GPLHR_OK) conv[i] = converged_update(c);
    });
  }
  for (int i = 0; i < nctx; ++i) {
    ctxs[i]->num_sms = saved_sms[i];
    ctxs[i]->tc = saved_tc[i] != 0;
    ctxs[i]->pk_work = nullptr;
    if (fatal != GPLHR_OK && st[i] == GPLHR_OK && !conv[i]) {
      st[i] = fatal;
      ctxs[i]->err = R.err;
    }
  }
  return fatal;
}

// ------------------------------------------------------------ GPLHR-EIG ------
// Algorithm 3 (Appendix A): the eigenvector-based variant.  The iterate X has unit
// columns; its Rayleigh quotients alpha_j / beta_j (bilinear forms x^* A x, x^* B x) are
// the eigenvalue approximations; the trial and test subspaces are built as in Algorithm 2
// with diag(beta), diag(alpha) in place of M_B, M_A; the projected pair is solved by its
// eigenvectors (ordered complex QZ, back substitution on the leading 2k block), which
// give X = Z Y(:, 1:k) and P (step 25, LOBPCG style, or step 27, thick restart).

// Upload the k x 2k row-major matrices [diag(d), diag(d)] of the two coefficient vectors
// (residual stored and its column norms taken in one combination).
gplhr_status eig_upload_diag2(gplhr_ctx* ctx, double2* dst, const std::vector<cd>& d, double2* stage) {
  const int k = ctx->k;
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < 2 * k; ++j) stage[i * 2 * k + j] = (j % k == i) ? d2(d[i]) : make_double2(0.0, 0.0);
  return upload(ctx, dst, stage, (size_t)2 * k * k);
}

// Step 28 (and steps 1-2): x_j <- x_j / ||x_j||, A X, B X, alpha, beta, Q <- (A - sigma B) X
// (U's first k columns), the residual R = A X diag(beta) - B X diag(alpha) into Rw with
// its column norms; the host receives alpha, beta and the backward errors.
gplhr_status eig_refresh(gplhr_ctx* ctx) {
  const int k = ctx->k, sm = ctx->s_max;
  const Blk none{nullptr, 0};
  const Blk X{ctx->eX, k}, AX{ctx->eAX, k}, BX{ctx->hasB ? ctx->eBX : ctx->eX, k};
  TRY(gram(ctx, X, k, X, k, none, 0, ctx->dGram));
  std::vector<double2> G((size_t)k * k);
  CK(cudaMemcpyAsync(G.data(), ctx->dGram, (size_t)k * k * sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  double2* hs = ctx->h_small;
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) {
      const double nj = std::sqrt(G[(size_t)j * k + j].x);
      hs[i * k + j] = make_double2(i == j && nj > 0.0 ? 1.0 / nj : 0.0, 0.0);
    }
  TRY(upload(ctx, ctx->dC1, hs, (size_t)k * k));
  TRY(combine(ctx, {In{X, k, ctx->dC1, kOne}}, X, k, false, nullptr, none, -1, -1, true, 0));
  TRY(spmm_AB(ctx, X, k, AX, ctx->hasB ? BX : none));
  TRY(gram(ctx, X, k, AX, k, BX, k, ctx->dPhiPsi));
  std::vector<double2> H((size_t)k * 2 * k);
  CK(cudaMemcpyAsync(H.data(), ctx->dPhiPsi, H.size() * sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->ea.assign(k, cd(0.0, 0.0));
  ctx->eb.assign(k, cd(0.0, 0.0));
  for (int j = 0; j < k; ++j) {
    ctx->ea[j] = cd(H[(size_t)j * 2 * k + j].x, H[(size_t)j * 2 * k + j].y);
    ctx->eb[j] = cd(H[(size_t)j * 2 * k + k + j].x, H[(size_t)j * 2 * k + k + j].y);
  }
  const int ph = prof_begin(ctx, KC_OTHER, 8.0 * ctx->n * k, 48.0 * ctx->n * k);
  gplhr::axpby_kernel<<<grid_for((size_t)ctx->n * k, 256, 8 * ctx->num_sms), 256, 0, ctx->stream>>>(
      ctx->n, k, kOne, ctx->eAX, k, d2(-ctx->sigma), BX.p, k, ctx->U, sm);
  prof_end(ctx, ph);
  CK(cudaGetLastError());
  TRY(eig_upload_diag2(ctx, ctx->dC1, ctx->eb, ctx->h_small));
  TRY(eig_upload_diag2(ctx, ctx->dC2, ctx->ea, ctx->h_small + 2 * k * k));
  TRY(combine(ctx, {In{AX, k, ctx->dC1, kOne}, In{BX, k, ctx->dC2, kMinusOne}}, Blk{ctx->Rw, k}, 2 * k, false,
              nullptr, none, k, k));
  CK(cudaMemcpyAsync(ctx->h_norms, ctx->d_norms, k * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(ctx->h_diag, ctx->d_diag, 3 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->resid.assign(k, 0.0);
  for (int j = 0; j < k; ++j) {
    const double den = std::abs(ctx->eb[j]) * ctx->normA + std::abs(ctx->ea[j]) * ctx->normB;
    ctx->resid[j] = std::sqrt(ctx->h_norms[j]) / den;
    if (!std::isfinite(ctx->resid[j])) {
      ctx->err = "non-finite residual";
      return GPLHR_ENUMERIC;
    }
  }
  if (ctx->h_diag[1] != 0) {
    ctx->err = "orth(): Cholesky QR broke down even with the shifted first pass";
    return GPLHR_ESINGULAR;
  }
  if (ctx->h_diag[2] != 0) {
    ctx->err = "tensor-core product: wait for completion gave up";
    return GPLHR_ETIMEOUT;
  }
  return GPLHR_OK;
}

gplhr_status eig_start(gplhr_ctx* ctx) {
  const int k = ctx->k;
  ctx->it = 0;
  ctx->q = 0;
  ctx->m = ctx->m0;
  ctx->hasP = false;
  ctx->n_spmm = ctx->n_prec = ctx->n_qz = ctx->n_inner = 0;
  ctx->h2d_bytes = ctx->d2h_bytes = 0;
  ctx->bulk32 = false;
  CK(cudaMemsetAsync(ctx->d_diag, 0, 3 * sizeof(int), ctx->stream));
  gplhr::copy_block_kernel<<<grid_for((size_t)ctx->n * k, 256, 8 * ctx->num_sms), 256, 0, ctx->stream>>>(
      ctx->n, k, ctx->Z, ctx->s_max, ctx->eX, k);
  CK(cudaGetLastError());
  TRY(eig_refresh(ctx));
  ctx->started = true;
  return GPLHR_OK;
}

gplhr_status eig_iterate_once(gplhr_ctx* ctx) {
  const int k = ctx->k, m = ctx->m0, sm = ctx->s_max;
  const Blk none{nullptr, 0};
  const Blk V = blkZ(ctx, 0), Q = blkU(ctx, 0);
  const Blk right = ctx->hasB ? Q : V;
  // step 4: V = orth(X), Q = orth((A - sigma B) X)
  gplhr::copy_block_kernel<<<grid_for((size_t)ctx->n * k, 256, 8 * ctx->num_sms), 256, 0, ctx->stream>>>(
      ctx->n, k, ctx->eX, k, ctx->Z, sm);
  CK(cudaGetLastError());
  TRY(orth_against(ctx, none, 0, V, k));
  TRY(orth_against(ctx, none, 0, Q, k));
  TRY(spmm_AB(ctx, V, k, blkAZ(ctx, 0), blkBZ(ctx, 0)));  // A V, B V: the pencil's first k columns
  // steps 5-10: W from the residual A X diag(beta) - B X diag(alpha) (in Rw)
  Blk R{ctx->Rw, k};
  TRY(project_out(ctx, right, k, R, k));
  TRY(precond_apply(ctx, R, k, blkZ(ctx, k)));
  TRY(orth_against(ctx, V, k, blkZ(ctx, k), k));
  TRY(spmm_AB(ctx, blkZ(ctx, k), k, blkAZ(ctx, k), blkBZ(ctx, k)));
  // steps 11-18
  if (m > 0) {
    double2* hm = ctx->h_small + 4 * k * k;
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) {
        hm[i * k + j] = i == j ? d2(ctx->eb[i]) : make_double2(0.0, 0.0);
        hm[k * k + i * k + j] = i == j ? d2(ctx->ea[i]) : make_double2(0.0, 0.0);
      }
    TRY(upload(ctx, ctx->dMBa, hm, 2 * k * k));
  }
  for (int l = 1; l <= m; ++l) {
    const int prev = l * k, cur = (l + 1) * k;
    TRY(combine(ctx, {In{blkAZ(ctx, prev), k, ctx->dMBa, kOne}, In{blkBZ(ctx, prev), k, ctx->dMBa + k * k, kMinusOne}},
                R, k, false));
    TRY(project_out(ctx, right, k, R, k));
    TRY(precond_apply(ctx, R, k, blkZ(ctx, cur)));
    TRY(orth_against(ctx, V, cur, blkZ(ctx, cur), k));
    TRY(spmm_AB(ctx, blkZ(ctx, cur), k, blkAZ(ctx, cur), blkBZ(ctx, cur)));
  }
  // step 19: P against V, W, S, orth; A P, B P by sparse products
  const int pslot = (m + 2) * k;
  int s = pslot;
  if (ctx->hasP) {
    gplhr::copy_block_kernel<<<grid_for((size_t)ctx->n * k, 256, 8 * ctx->num_sms), 256, 0, ctx->stream>>>(
        ctx->n, k, ctx->Pb, k, ctx->Z + pslot, sm);
    CK(cudaGetLastError());
    TRY(orth_against(ctx, V, pslot, blkZ(ctx, pslot), k));
    TRY(spmm_AB(ctx, blkZ(ctx, pslot), k, blkAZ(ctx, pslot), blkBZ(ctx, pslot)));
    s += k;
  }
  const int sk = s - k;
  // steps 20-22: Qhat = orth((A - sigma B) [W S P]) against Q; U = [Q Qhat]
  const int ph = prof_begin(ctx, KC_OTHER, 8.0 * ctx->n * sk, 48.0 * ctx->n * sk);
  gplhr::axpby_kernel<<<grid_for((size_t)ctx->n * sk, 256, 8 * ctx->num_sms), 256, 0, ctx->stream>>>(
      ctx->n, sk, kOne, ctx->AZ + k, sm, d2(-ctx->sigma), blkBZ(ctx, k).p, sm, ctx->U + k, sm);
  prof_end(ctx, ph);
  CK(cudaGetLastError());
  TRY(orth_against(ctx, Q, k, blkU(ctx, k), sk));
  // step 23: eigenvectors of (U^* A Z, U^* B Z) nearest sigma
  TRY(gram(ctx, blkU(ctx, 0), s, blkAZ(ctx, 0), s, blkBZ(ctx, 0), s, ctx->dPhiPsi));
  ctx->d2h_bytes += (int64_t)2 * s * s * sizeof(double2);
  CK(cudaMemcpyAsync(ctx->h_phipsi, ctx->dPhiPsi, (size_t)2 * s * s * sizeof(double2), cudaMemcpyDeviceToHost,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  SqMat RAb, RBb, YLb, YRb;
  TRY(host_qz(ctx, s, RAb, RBb, YLb, YRb, 2 * k, 0, 2 * k));
  SqMat RA2(2 * k), RB2(2 * k);
  for (int i = 0; i < 2 * k; ++i)
    for (int j = 0; j < 2 * k; ++j) {
      RA2(i, j) = RAb(i, j);
      RB2(i, j) = RBb(i, j);
    }
  const SqMat Zt = gplhr::tri_eigvecs(RA2, RB2);
  // Y = Ybar_R(:, 1:2k) Zt, unit columns; staged as Y(:, 1:k) and Y(:, k+1:2k), s x k each
  double2* hy = ctx->h_small + 6 * k * k;
  double2* hp = hy + (size_t)s * k;
  for (int j = 0; j < 2 * k; ++j) {
    std::vector<cd> col(s, cd(0.0, 0.0));
    double nrm = 0.0;
    for (int i = 0; i < s; ++i) {
      cd acc(0.0, 0.0);
      for (int t = 0; t <= j; ++t) acc += YRb(i, t) * Zt(t, j);
      col[i] = acc;
      nrm += std::norm(acc);
    }
    nrm = std::sqrt(nrm);
    for (int i = 0; i < s; ++i) (j < k ? hy : hp)[(size_t)i * k + (j % k)] = d2(col[i] / nrm);
  }
  TRY(upload(ctx, ctx->dYR, hy, (size_t)s * k));
  TRY(upload(ctx, ctx->dYL, hp, (size_t)s * k));
  // steps 24-27: X = Z Y(:, 1:k); P = [W S P] Y(k+1:s, 1:k) (step 25) or Z Y(:, k+1:2k) (27)
  TRY(combine(ctx, {In{blkZ(ctx, 0), s, ctx->dYR, kOne}}, Blk{ctx->eX, k}, k, false));
  if (ctx->p_mode == 1)
    TRY(combine(ctx, {In{blkZ(ctx, k), sk, ctx->dYR + (size_t)k * k, kOne}}, Blk{ctx->Pb, k}, k, false));
  else
    TRY(combine(ctx, {In{blkZ(ctx, 0), s, ctx->dYL, kOne}}, Blk{ctx->Pb, k}, k, false));
  ctx->hasP = true;
  ctx->it += 1;
  return eig_refresh(ctx);  // step 28
}

gplhr_status eig_run(gplhr_ctx* ctx, int niter, gplhr_info* info, bool* conv_out) {
  auto all = [&]() {
    for (double r : ctx->resid)
      if (!(r <= ctx->tol)) return false;
    return !ctx->resid.empty();
  };
  bool conv = all();
  for (int i = 0; i < niter && !conv; ++i) {
    TRY(eig_iterate_once(ctx));
    conv = all();
  }
  fill_info(ctx, info);
  if (conv_out) *conv_out = conv;
  return GPLHR_OK;
}

// ------------------------------------------------------------------ setup ----

// Checks a CSR descriptor; rp / ci point at its row pointers and column indices on the host
// (the caller's arrays, or copies in rpv / civ when they live on the device).  The rows are
// checked in a fixed number of ranges on host threads; the lowest failing range's error is
// the one reported.
gplhr_status validate_csr(const gplhr_csr* M, int64_t n, std::string& err, std::vector<int>& rpv,
                          std::vector<int>& civ, const int*& rp, const int*& ci) {
  if (!M || M->n != n || M->nnz < 0 || !M->rowptr || (M->nnz > 0 && (!M->colind || !M->vals))) {
    err = "invalid CSR descriptor";
    return GPLHR_EINVAL;
  }
  if (M->dtype != GPLHR_R64 && M->dtype != GPLHR_C128) {
    err = "CSR dtype must be GPLHR_R64 or GPLHR_C128";
    return GPLHR_EINVAL;
  }
  if (M->on_device) {
    rpv.resize(n + 1);
    civ.resize(M->nnz);
    if (cudaMemcpy(rpv.data(), M->rowptr, (n + 1) * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
        (M->nnz > 0 &&
         cudaMemcpy(civ.data(), M->colind, M->nnz * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)) {
      err = "cannot read device CSR arrays";
      return GPLHR_ECUDA;
    }
    rp = rpv.data();
    ci = civ.data();
  } else {
    rp = static_cast<const int*>(M->rowptr);
    ci = static_cast<const int*>(M->colind);
  }
  if (rp[0] != 0 || rp[n] != M->nnz) {
    err = "CSR rowptr must start at 0 and end at nnz";
    return GPLHR_EINVAL;
  }
  const int parts = M->nnz < (int64_t)1 << 20 ? 1 : 8;
  std::vector<int> bad(parts, 0);  // 1: rowptr not monotone, 2: column indices
  auto work = [&](int p) {
    const int64_t r0 = n * p / parts, r1 = n * (p + 1) / parts;
    for (int64_t i = r0; i < r1 && !bad[p]; ++i) {
      if (rp[i + 1] < rp[i] || rp[i + 1] > M->nnz) {  // (no index beyond nnz is read)
        bad[p] = 1;
        break;
      }
      for (int j = rp[i]; j < rp[i + 1]; ++j)
        if (ci[j] < 0 || ci[j] >= n || (j > rp[i] && ci[j] <= ci[j - 1])) {
          bad[p] = 2;
          break;
        }
    }
  };
  std::vector<std::thread> pool;
  for (int p = 1; p < parts; ++p) pool.emplace_back(work, p);
  work(0);
  for (auto& t : pool) t.join();
  for (int p = 0; p < parts; ++p) {
    if (bad[p] == 1) {
      err = "CSR rowptr not monotone or beyond nnz";
      return GPLHR_EINVAL;
    }
    if (bad[p] == 2) {
      err = "CSR column indices out of range or not strictly increasing in a row";
      return GPLHR_EINVAL;
    }
  }
  return GPLHR_OK;
}

// max_j sum_i |m_ij| over a CSR matrix: a fixed number of row ranges, one per host thread,
// each summing its columns into its own array; the arrays are then added in range order, so
// the result does not depend on the scheduling.
double csr_onenorm(int64_t n, int64_t nnz, const int* rp, const int* ci, const double* vals, bool cplx) {
  const int parts = nnz < (int64_t)1 << 20 ? 1 : 8;
  std::vector<std::vector<double>> part(parts, std::vector<double>(n, 0.0));
  auto work = [&](int p) {
    const int64_t r0 = n * p / parts, r1 = n * (p + 1) / parts;
    std::vector<double>& cs = part[p];
    for (int64_t r = r0; r < r1; ++r)
      for (int64_t e = rp[r]; e < rp[r + 1]; ++e)
        cs[ci[e]] += cplx ? std::hypot(vals[2 * e], vals[2 * e + 1]) : std::fabs(vals[e]);
  };
  std::vector<std::thread> pool;
  for (int p = 1; p < parts; ++p) pool.emplace_back(work, p);
  work(0);
  for (auto& t : pool) t.join();
  double mx = 0.0;
  for (int64_t c = 0; c < n; ++c) {
    double v = 0.0;
    for (int p = 0; p < parts; ++p) v += part[p][c];
    mx = std::max(mx, v);
  }
  return mx;
}

gplhr_status upload_csr(gplhr_ctx* ctx, const gplhr_csr* M, DevCsr& D, double* onenorm) {
  std::vector<int> rpv, civ;
  const int *rp = nullptr, *ci = nullptr;
  gplhr_status st = validate_csr(M, ctx->n, ctx->err, rpv, civ, rp, ci);
  if (st != GPLHR_OK) return st;
  const int64_t n = ctx->n, nnz = M->nnz;
  const size_t vsz = M->dtype == GPLHR_C128 ? 16 : 8;
  D.dtype = M->dtype;
  D.nnz = nnz;
  CK(cudaMalloc(&D.rowptr, (n + 1) * sizeof(int)));
  CK(cudaMalloc(&D.col, std::max<int64_t>(nnz, 1) * sizeof(int)));
  CK(cudaMalloc(&D.val, std::max<int64_t>(nnz, 1) * vsz));
  CK(cudaMemcpy(D.rowptr, rp, (n + 1) * sizeof(int), cudaMemcpyHostToDevice));
  if (nnz > 0) {
    CK(cudaMemcpy(D.col, ci, nnz * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(D.val, M->vals, nnz * vsz, M->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice));
  }
  if (onenorm) {  // ||M||_1 = max column sum of |m_ij|, on the host
    std::vector<double> dvals;
    const double* vals = static_cast<const double*>(M->vals);
    if (M->on_device) {
      dvals.resize(nnz * (vsz / 8));
      if (nnz > 0) CK(cudaMemcpy(dvals.data(), D.val, nnz * vsz, cudaMemcpyDeviceToHost));
      vals = dvals.data();
    }
    *onenorm = csr_onenorm(n, nnz, rp, ci, vals, vsz == 16);
  }
  return GPLHR_OK;
}

template <typename VTA, typename VTB>
void launch_prec_setup(gplhr_ctx* ctx, int kind, double2* out, int nblocks) {
  gplhr::CsrDev<VTA> a{ctx->A.rowptr, ctx->A.col, (const VTA*)ctx->A.val};
  gplhr::CsrDev<VTB> b{ctx->B.rowptr, ctx->B.col, (const VTB*)ctx->B.val};
  const double2 sg = d2(ctx->sigma);
  if (kind == GPLHR_PREC_JACOBI)
    gplhr::jacobi_setup_kernel<VTA, VTB><<<(ctx->n + 255) / 256, 256, 0, ctx->stream>>>(ctx->n, a, b, ctx->hasB,
                                                                                        sg, out);
  else
    gplhr::extract_blocks_kernel<VTA, VTB><<<(nblocks * ctx->bs + 255) / 256, 256, 0, ctx->stream>>>(
        ctx->n, ctx->bs, a, b, ctx->hasB, sg, out, nblocks);
}

gplhr_status setup_preconditioner(gplhr_ctx* ctx, const gplhr_precond* T) {
  ctx->prec = T ? T->kind : GPLHR_PREC_NONE;
  if (ctx->prec == GPLHR_PREC_NONE) return GPLHR_OK;
  if (ctx->prec == GPLHR_PREC_CSR) {
    if (!T->T_csr || T->T_csr->dtype != GPLHR_C128) {
      ctx->err = "CSR preconditioner needs a complex (GPLHR_C128) matrix";
      return GPLHR_EINVAL;
    }
    return upload_csr(ctx, T->T_csr, ctx->Tcsr, nullptr);
  }
  if (ctx->prec != GPLHR_PREC_JACOBI && ctx->prec != GPLHR_PREC_BLOCK_JACOBI) {
    ctx->err = "unknown preconditioner kind";
    return GPLHR_EINVAL;
  }
  ctx->bs = ctx->prec == GPLHR_PREC_JACOBI ? 1 : T->block_size;
  if (ctx->bs < 1 || ctx->bs > 32) {
    ctx->err = "block-Jacobi block size must be in [1, 32]";
    return GPLHR_EINVAL;
  }
  const int n = ctx->n, bs = ctx->bs;
  const int nblocks = (n + bs - 1) / bs;
  const size_t elems = ctx->prec == GPLHR_PREC_JACOBI ? (size_t)n : (size_t)nblocks * bs * bs;
  CK(cudaMalloc(&ctx->prec_data, elems * sizeof(double2)));
  const int ta = ctx->A.dtype, tb = ctx->hasB ? ctx->B.dtype : GPLHR_R64;
  if (ta == GPLHR_R64 && tb == GPLHR_R64) launch_prec_setup<double, double>(ctx, ctx->prec, ctx->prec_data, nblocks);
  else if (ta == GPLHR_R64) launch_prec_setup<double, double2>(ctx, ctx->prec, ctx->prec_data, nblocks);
  else if (tb == GPLHR_R64) launch_prec_setup<double2, double>(ctx, ctx->prec, ctx->prec_data, nblocks);
  else launch_prec_setup<double2, double2>(ctx, ctx->prec, ctx->prec_data, nblocks);
  CK(cudaGetLastError());
  if (ctx->prec == GPLHR_PREC_JACOBI) {
    std::vector<double2> d(n);
    CK(cudaMemcpyAsync(d.data(), ctx->prec_data, n * sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    double amax = 0.0, spread = 0.0;
    bool zero = false;
    for (int i = 0; i < n; ++i) {
      amax = std::max(amax, std::hypot(d[i].x, d[i].y));
      spread = std::max(spread, std::hypot(d[i].x - d[0].x, d[i].y - d[0].y));
      zero = zero || (d[i].x == 0.0 && d[i].y == 0.0);
    }
    if (amax == 0.0 || spread <= 1e-12 * amax) {  // constant diagonal: T is a multiple of I
      ctx->prec = GPLHR_PREC_NONE;
      cudaFree(ctx->prec_data);
      ctx->prec_data = nullptr;
      return GPLHR_OK;
    }
    if (zero) {
      ctx->err = "Jacobi: zero diagonal entry of A - sigma B";
      return GPLHR_ESINGULAR;
    }
    gplhr::reciprocal_kernel<<<(n + 255) / 256, 256, 0, ctx->stream>>>(n, ctx->prec_data);
    CK(cudaGetLastError());
    return GPLHR_OK;
  }
  int* dflag = ctx->d_status;
  CK(cudaMemsetAsync(dflag, 0, sizeof(int), ctx->stream));
  const int wpc = 4;
  const size_t smem = (size_t)wpc * bs * 2 * bs * sizeof(double2);
  gplhr::invert_blocks_kernel<<<(nblocks + wpc - 1) / wpc, 32 * wpc, smem, ctx->stream>>>(nblocks, bs,
                                                                                         ctx->prec_data, dflag);
  CK(cudaGetLastError());
  int flag = 0;
  CK(cudaMemcpyAsync(&flag, dflag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (flag != 0) {
    ctx->err = "block-Jacobi: singular diagonal block " + std::to_string(flag - 1) + " of A - sigma B";
    return GPLHR_ESINGULAR;
  }
  return GPLHR_OK;
}

// FP32 copies used by the bulk phase of the mixed mode: matrix values, block-Jacobi
// inverse blocks, and a complex64 staging block for the sparse products' input.
gplhr_status to_fp32(gplhr_ctx* ctx, const void* src, size_t count, void** dst) {
  std::vector<double> h(count);
  std::vector<float> f(count);
  CK(cudaMemcpy(h.data(), src, count * sizeof(double), cudaMemcpyDeviceToHost));
  for (size_t i = 0; i < count; ++i) f[i] = (float)h[i];
  CK(cudaMalloc(dst, std::max<size_t>(count, 1) * sizeof(float)));
  CK(cudaMemcpy(*dst, f.data(), count * sizeof(float), cudaMemcpyHostToDevice));
  return GPLHR_OK;
}

gplhr_status make_fp32_copies(gplhr_ctx* ctx) {
  auto vals = [](const DevCsr& D) { return (size_t)D.nnz * (D.dtype == GPLHR_C128 ? 2 : 1); };
  TRY(to_fp32(ctx, ctx->A.val, vals(ctx->A), &ctx->A.val32));
  if (ctx->hasB) TRY(to_fp32(ctx, ctx->B.val, vals(ctx->B), &ctx->B.val32));
  if (ctx->prec == GPLHR_PREC_CSR) TRY(to_fp32(ctx, ctx->Tcsr.val, vals(ctx->Tcsr), &ctx->Tcsr.val32));
  if (ctx->prec == GPLHR_PREC_BLOCK_JACOBI) {
    const size_t nb = (size_t)((ctx->n + ctx->bs - 1) / ctx->bs) * ctx->bs * ctx->bs;
    void* p = nullptr;
    TRY(to_fp32(ctx, ctx->prec_data, 2 * nb, &p));
    ctx->prec32 = (float2*)p;
  }
  CK(cudaMalloc(&ctx->X32, (size_t)ctx->n * ((ctx->k + 1) & ~1) * sizeof(float2)));
  return GPLHR_OK;
}

void free_all(gplhr_ctx* c) {
  auto F = [](void* p) {
    if (p) cudaFree(p);
  };
  F(c->dV1); F(c->dQ1); F(c->eX); F(c->eAX); F(c->eBX);
  F(c->A.rowptr); F(c->A.col); F(c->A.val); F(c->A.val32);
  F(c->B.rowptr); F(c->B.col); F(c->B.val); F(c->B.val32);
  F(c->Tcsr.rowptr); F(c->Tcsr.col); F(c->Tcsr.val); F(c->Tcsr.val32);
  F(c->prec_data); F(c->prec32); F(c->X32);
  F(c->Z); F(c->AZ); F(c->BZ); F(c->U); F(c->Pb); F(c->APb); F(c->BPb);
  F(c->Rw); F(c->Tw1); F(c->Tw2); F(c->Tw3);
  F(c->dC1); F(c->dC2); F(c->dMBa); F(c->dMAa); F(c->dYR); F(c->dYL); F(c->dPhiPsi); F(c->dGram);
  F(c->dProjC); F(c->dRinv); F(c->dTrackC); F(c->dTrackR); F(c->gram_part); F(c->norm_part); F(c->d_norms); F(c->d_status); F(c->d_diag);
  F(c->gmV); F(c->gmT); F(c->gmAX); F(c->gmBX); F(c->gmY);
  if (c->h_gm) cudaFreeHost(c->h_gm);
  if (c->h_gm_status) cudaFreeHost(c->h_gm_status);
  if (c->h_gmY) cudaFreeHost(c->h_gmY);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  if (c->h_small) cudaFreeHost(c->h_small);
  if (c->h_phipsi) cudaFreeHost(c->h_phipsi);
  if (c->h_norms) cudaFreeHost(c->h_norms);
  if (c->h_diag) cudaFreeHost(c->h_diag);
  if (c->h_track) cudaFreeHost(c->h_track);
  if (c->h_status) cudaFreeHost(c->h_status);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
}

gplhr_status allocate(gplhr_ctx* ctx) {
  const size_t n = ctx->n, k = ctx->k, sm = ctx->s_max;
  const size_t nb = n * sm * sizeof(double2);
  CK(cudaMalloc(&ctx->Z, nb));
  CK(cudaMalloc(&ctx->AZ, nb));
  if (ctx->hasB) CK(cudaMalloc(&ctx->BZ, nb));
  CK(cudaMalloc(&ctx->U, nb));
  const size_t kb = n * k * sizeof(double2);
  CK(cudaMalloc(&ctx->Pb, kb));
  CK(cudaMalloc(&ctx->APb, kb));
  if (ctx->hasB) CK(cudaMalloc(&ctx->BPb, kb));
  CK(cudaMalloc(&ctx->Rw, kb));
  CK(cudaMalloc(&ctx->Tw1, kb));
  CK(cudaMalloc(&ctx->Tw2, kb));
  CK(cudaMalloc(&ctx->Tw3, kb));
  CK(cudaMemset(ctx->Z, 0, nb));
  CK(cudaMemset(ctx->AZ, 0, nb));
  CK(cudaMemset(ctx->U, 0, nb));
  if (ctx->hasB) CK(cudaMemset(ctx->BZ, 0, nb));
  const size_t s2 = sm * sm * sizeof(double2);
  CK(cudaMalloc(&ctx->dC1, 2 * k * k * sizeof(double2)));
  CK(cudaMalloc(&ctx->dC2, 2 * k * k * sizeof(double2)));
  CK(cudaMalloc(&ctx->dMBa, 2 * k * k * sizeof(double2)));
  CK(cudaMalloc(&ctx->dMAa, k * k * sizeof(double2)));
  CK(cudaMalloc(&ctx->dYR, 2 * s2));
  CK(cudaMalloc(&ctx->dYL, 2 * s2));
  CK(cudaMalloc(&ctx->dPhiPsi, 2 * s2));
  CK(cudaMalloc(&ctx->dGram, 2 * s2));
  ctx->trk = std::max(sm * sm, (size_t)ctx->gm_steps * k * k);
  CK(cudaMalloc(&ctx->dProjC, std::max(2 * s2, ctx->trk * sizeof(double2))));
  CK(cudaMalloc(&ctx->dRinv, 3 * s2));
  CK(cudaMalloc(&ctx->dTrackC, 3 * ctx->trk * sizeof(double2)));
  CK(cudaMalloc(&ctx->dTrackR, 3 * s2));
  CK(cudaMallocHost(&ctx->h_track, 6 * s2));
  CK(cudaMallocHost(&ctx->h_status, 4 * sizeof(int)));
  ctx->gram_part_elems = (size_t)(4 * ctx->num_sms + 8) * gplhr::GRAM_THREADS * 8;
  ctx->gram_part_elems = std::max(ctx->gram_part_elems, 2 * sm * sm);
  CK(cudaMalloc(&ctx->gram_part, ctx->gram_part_elems * sizeof(double2)));
  CK(cudaMalloc(&ctx->norm_part, (size_t)(4 * ctx->num_sms + 8) * gplhr::COMB_MAX_NORMS * sizeof(double)));
  CK(cudaMalloc(&ctx->d_norms, gplhr::COMB_MAX_NORMS * sizeof(double)));
  CK(cudaMalloc(&ctx->d_status, 8 * sizeof(int)));
  CK(cudaMalloc(&ctx->d_diag, 3 * sizeof(int)));
  CK(cudaMemset(ctx->d_diag, 0, 3 * sizeof(int)));
  CK(cudaMallocHost(&ctx->h_small, (8 * k * k + 4 * sm * sm) * sizeof(double2)));
  CK(cudaMallocHost(&ctx->h_phipsi, 2 * s2));
  CK(cudaMallocHost(&ctx->h_norms, gplhr::COMB_MAX_NORMS * sizeof(double)));
  CK(cudaMallocHost(&ctx->h_diag, 3 * sizeof(int)));
  ctx->h_diag[0] = ctx->h_diag[1] = ctx->h_diag[2] = 0;
  if (ctx->gm_steps > 0) {
    const size_t gs = ctx->gm_steps;
    CK(cudaMalloc(&ctx->gmV, n * (gs + 1) * k * sizeof(double2)));
    CK(cudaMalloc(&ctx->gmT, kb));
    CK(cudaMalloc(&ctx->gmAX, kb));
    if (ctx->hasB) CK(cudaMalloc(&ctx->gmBX, kb));
    CK(cudaMalloc(&ctx->gmY, gs * k * k * sizeof(double2)));
    CK(cudaMallocHost(&ctx->h_gm, (gs + 1) * (3 * ctx->trk + 3 * k * k) * sizeof(double2)));
    CK(cudaMallocHost(&ctx->h_gm_status, (gs + 1) * sizeof(int)));
    CK(cudaMallocHost(&ctx->h_gmY, gs * k * k * sizeof(double2)));
  }
  return GPLHR_OK;
}

gplhr_status set_smem_limits(gplhr_ctx* ctx) {
  const int big = (int)kCombSmemMax;
  CK(cudaFuncSetAttribute(gplhr::combine_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  CK(cudaFuncSetAttribute(gplhr::combine_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  CK(cudaFuncSetAttribute(gplhr::gram_partial_kernel<8, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  CK(cudaFuncSetAttribute(gplhr::gram_partial_kernel<4, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  CK(cudaFuncSetAttribute(gplhr::gram_partial_kernel<2, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  CK(cudaFuncSetAttribute(gplhr::gram_partial_kernel<1, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  CK(cudaFuncSetAttribute(gplhr::gram_partial_x32_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  CK(cudaFuncSetAttribute(gplhr::gram_partial_x32_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  CK(cudaFuncSetAttribute(gplhr::gram_partial_x32_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  CK(cudaFuncSetAttribute(gplhr::gram_partial_x32_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  CK(cudaFuncSetAttribute(gplhr::gram_partial_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  CK(cudaFuncSetAttribute(gplhr::gram_partial_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  CK(cudaFuncSetAttribute(gplhr::gram_partial_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  CK(cudaFuncSetAttribute(gplhr::gram_partial_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  CK(cudaFuncSetAttribute(gplhr::chol_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  CK(cudaFuncSetAttribute(gplhr::block_jacobi_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  CK(cudaFuncSetAttribute(gplhr::block_jacobi_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  CK(cudaFuncSetAttribute(gplhr::block_jacobi_kernel<float, float2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          big));
  CK(cudaFuncSetAttribute(gplhr::invert_blocks_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  CK(cudaFuncSetAttribute(gplhr::tc_combine_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  CK(cudaFuncSetAttribute(gplhr::tc_combine_kernel<2, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  CK(cudaFuncSetAttribute(gplhr::tc_combine_kernel<4, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  CK(cudaFuncSetAttribute(gplhr::tc_combine_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  CK(cudaFuncSetAttribute(gplhr::tc_combine_kernel<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  CK(cudaFuncSetAttribute(gplhr::tc_combine_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  CK(cudaFuncSetAttribute(gplhr::tc_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)gplhr::tg_smem_bytes(2, 64)));
  CK(cudaFuncSetAttribute(gplhr::tc_gram_wide_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)kTwSmemMax));
  CK(cudaFuncSetAttribute(gplhr::tc_gram_narrow_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  CK(cudaFuncSetAttribute(gplhr::tc_gram_narrow_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  return GPLHR_OK;
}

gplhr_status load_V0(gplhr_ctx* ctx, const void* V0, int where, int is_complex, uint64_t seed) {
  const int n = ctx->n, k = ctx->k;
  if (!V0) {
    gplhr::gaussian_block_kernel<<<grid_for((size_t)n * k, 256, 8 * ctx->num_sms), 256, 0, ctx->stream>>>(
        n, k, seed, ctx->Z, ctx->s_max);
    CK(cudaGetLastError());
    return GPLHR_OK;
  }
  const cudaMemcpyKind kind = where == GPLHR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (is_complex && where == GPLHR_DEVICE) {
    CK(cudaMemcpy2DAsync(ctx->Z, ctx->s_max * sizeof(double2), V0, k * sizeof(double2), k * sizeof(double2), n,
                         kind, ctx->stream));
  } else if (is_complex) {  // one contiguous copy from the host, then spread to the row stride of Z
    CK(cudaMemcpyAsync(ctx->Tw1, V0, (size_t)n * k * sizeof(double2), kind, ctx->stream));
    gplhr::copy_block_kernel<<<grid_for((size_t)n * k, 256, 8 * ctx->num_sms), 256, 0, ctx->stream>>>(
        n, k, ctx->Tw1, k, ctx->Z, ctx->s_max);
    CK(cudaGetLastError());
  } else {
    CK(cudaMemcpyAsync(ctx->Tw1, V0, (size_t)n * k * sizeof(double), kind, ctx->stream));
    gplhr::real_to_complex_kernel<<<grid_for((size_t)n * k, 256, 8 * ctx->num_sms), 256, 0, ctx->stream>>>(
        n, k, (const double*)ctx->Tw1, ctx->Z, ctx->s_max);
    CK(cudaGetLastError());
  }
  return GPLHR_OK;
}

bool valid_block(const void* p, int ld, int w) { return p != nullptr && w >= 0 && ld >= w; }

}  // namespace

// ------------------------------------------------------- allocation-free Gram --
// Scratch of gplhr_gram_noalloc: the split-n partial sums of the Gram product live
// in this file-scope device array (4 MiB) instead of memory from cudaMalloc.  Every
// GPU that loads the library holds it until the process exits, and all calls on a
// device share it.
constexpr size_t kNoallocScratchElems = (size_t)1 << 18;  // double2 elements
constexpr int kNoallocMaxOut = 16384;                     // wx * wy limit
constexpr int kNoallocMaxCols = 768;                      // wx + wy limit (staged rows)
constexpr int64_t kNoallocMaxRows = (int64_t)1 << 30;     // n limit (int row indices)
static __device__ __align__(256) double2 g_noalloc_scratch[kNoallocScratchElems];

constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mu;
double2* g_noalloc_ptr[kNoallocMaxDevices] = {nullptr};
int g_noalloc_sms[kNoallocMaxDevices] = {0};

// Once per device, with that device current: the device address of the scratch array
// (host code only has a host-side stand-in for the symbol, which must never be passed
// to a kernel) and the shared-memory opt-in of the Gram kernels.
gplhr_status noalloc_setup(double2** ptr, int* sms) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoallocMaxDevices) {
    g_create_error = "gplhr_gram_noalloc: no usable current CUDA device";
    return GPLHR_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      g_create_error = std::string("gplhr_gram_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
      return GPLHR_ECUDA;
    }
    int nsm = 0;
    e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int big = 200 * 1024;
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(gplhr::gram_partial_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(gplhr::gram_partial_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(gplhr::gram_partial_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(gplhr::gram_partial_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    if (e != cudaSuccess) {
      g_create_error = std::string("gplhr_gram_noalloc: device set-up: ") + cudaGetErrorString(e);
      return GPLHR_ECUDA;
    }
    g_noalloc_sms[dev] = nsm;
    g_noalloc_ptr[dev] = (double2*)p;
  }
  *ptr = g_noalloc_ptr[dev];
  *sms = g_noalloc_sms[dev];
  return GPLHR_OK;
}

// ====================================================================== C ABI ==

extern "C" {

gplhr_status gplhr_create(const gplhr_csr* A, const gplhr_csr* B, double sigma_re, double sigma_im, int32_t k,
                          int32_t m, const gplhr_precond* T, const gplhr_opts* opts, gplhr_ctx** out) {
  if (!out) {
    g_create_error = "out must not be NULL";
    return GPLHR_EINVAL;
  }
  *out = nullptr;
  if (!A || A->n < 1 || A->n > (int64_t)0x7fffffff / 2) {
    g_create_error = "A must be a CSR matrix with 1 <= n < 2^30";
    return GPLHR_EINVAL;
  }
  if (k < 1 || m < 0 || m > 20 || (int64_t)(m + 3) * k > A->n || !std::isfinite(sigma_re) ||
      !std::isfinite(sigma_im) || (B && B->n != A->n) || k > 32 || (m + 2) * k > 80) {
    g_create_error = "invalid sizes: need 1 <= k <= 32, 0 <= m <= 20, (m+2) k <= 80, (m+3) k <= n, finite sigma";
    return GPLHR_EINVAL;
  }
  gplhr_ctx* ctx = new (std::nothrow) gplhr_ctx();
  if (!ctx) {
    g_create_error = "out of host memory";
    return GPLHR_ENOMEM;
  }
  ctx->n = (int)A->n;
  ctx->k = k;
  ctx->m0 = m;
  ctx->m = m;
  ctx->s_max = (m + 3) * k;
  ctx->sigma = cd(sigma_re, sigma_im);
  ctx->hasB = B != nullptr;
  if (opts) {
    if (opts->tol > 0) ctx->tol = opts->tol;
    if (opts->maxit > 0) ctx->maxit = opts->maxit;
    ctx->lock = opts->no_lock == 0;
    ctx->stream = (cudaStream_t)opts->stream;
    ctx->mixed = opts->precision == GPLHR_MIXED;
    if (opts->switch_tol > 0) ctx->switch_tol = opts->switch_tol;
    if (opts->stall_iters != 0) ctx->stall_iters = opts->stall_iters;
    ctx->factored = opts->pencil == 0;
    ctx->tc = opts->fp64_gemm == 0;
    ctx->graphs = opts->graphs != 0;
    ctx->autotune = opts->autotune != 0;
    ctx->right_proj = opts->no_right_proj == 0;
    if (opts->wait_limit < 0) {
      g_create_error = "opts.wait_limit must be >= 0";
      delete ctx;
      return GPLHR_EINVAL;
    }
    if (opts->wait_limit > 0) ctx->tc_wait_tries = std::min(opts->wait_limit, gplhr::TC_WAIT_TRIES);
    ctx->tc_probe = opts->wait_probe != 0;
    if (opts->p_mode < 0 || opts->p_mode > 2) {
      g_create_error = "opts.p_mode must be 0 (thick), 1 (LOBPCG style) or 2 (none)";
      delete ctx;
      return GPLHR_EINVAL;
    }
    ctx->p_mode = opts->p_mode;
    ctx->eig = opts->variant == 1;
    if (opts->variant < 0 || opts->variant > 1 ||
        (ctx->eig && (opts->precision != GPLHR_FP64 || opts->p_mode == 2 || opts->no_right_proj != 0))) {
      g_create_error = "opts.variant must be 0 (Schur vectors, Alg. 2) or 1 (eigenvectors, Alg. 3); the "
                       "eigenvector variant runs in FP64 with p_mode 0 or 1 and the projector before T";
      delete ctx;
      return GPLHR_EINVAL;
    }
    if (opts->precision != GPLHR_FP64 && opts->precision != GPLHR_MIXED) {
      g_create_error = "opts.precision must be GPLHR_FP64 or GPLHR_MIXED";
      delete ctx;
      return GPLHR_EINVAL;
    }
  }
  ctx->gm_steps = T ? T->inner_steps : 0;
  if (ctx->gm_steps < 0 || ctx->gm_steps > 32 || ctx->gm_steps * k > 384) {
    g_create_error = "T.inner_steps must be in [0, 32] with inner_steps * k <= 384";
    delete ctx;
    return GPLHR_EINVAL;
  }
  const int products = opts ? opts->products : 0;
  if (products < 0 || products > 2) {
    g_create_error = "opts.products must be 0, 1 or 2";
    delete ctx;
    return GPLHR_EINVAL;
  }
  auto fail = [&](gplhr_status st) {
    g_create_error = ctx->err;
    free_all(ctx);
    delete ctx;
    return st;
  };
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    ctx->err = "no CUDA device";
    return fail(GPLHR_ECUDA);
  }
  if (!ctx->stream) {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
      ctx->err = "cudaStreamCreate failed";
      return fail(GPLHR_ECUDA);
    }
    ctx->own_stream = true;
  }
  gplhr_status st;
  if ((st = set_smem_limits(ctx)) != GPLHR_OK) return fail(st);
  if ((st = upload_csr(ctx, A, ctx->A, &ctx->normA)) != GPLHR_OK) return fail(st);
  if (ctx->hasB && (st = upload_csr(ctx, B, ctx->B, &ctx->normB)) != GPLHR_OK) return fail(st);
  if ((st = allocate(ctx)) != GPLHR_OK) return fail(st);
  if (ctx->eig) {
    const size_t bytes = (size_t)ctx->n * ctx->k * sizeof(double2);
    if (cudaMalloc(&ctx->eX, bytes) != cudaSuccess || cudaMalloc(&ctx->eAX, bytes) != cudaSuccess ||
        (ctx->hasB && cudaMalloc(&ctx->eBX, bytes) != cudaSuccess)) {
      ctx->err = "cudaMalloc failed (eigenvector variant buffers)";
      return fail(GPLHR_ENOMEM);
    }
  }
  if ((st = setup_preconditioner(ctx, T)) != GPLHR_OK) return fail(st);
  if (ctx->mixed && (st = make_fp32_copies(ctx)) != GPLHR_OK) return fail(st);
  {
    // flops per block column: sparse products of one column vs an s-wide combination
    const double spmm = ((ctx->A.dtype == GPLHR_C128 ? 8.0 : 4.0) * ctx->A.nnz +
                         (ctx->hasB ? (ctx->B.dtype == GPLHR_C128 ? 8.0 : 4.0) * ctx->B.nnz : 0.0)) /
                        ctx->n;
    const double comb = 8.0 * ctx->s_max * (ctx->hasB ? 2.0 : 1.0);
    ctx->recompute = products == 2 || (products == 0 && spmm < comb);
  }
  if (ctx->autotune && (st = autotune_spmm(ctx)) != GPLHR_OK) return fail(st);
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
    ctx->err = "setup failed on the device";
    return fail(GPLHR_ECUDA);
  }
  *out = ctx;
  return GPLHR_OK;
}

gplhr_status gplhr_start(gplhr_ctx* ctx, const void* V0, int32_t V0_where, int32_t is_complex, uint64_t seed) {
  if (!ctx) return GPLHR_EINVAL;
  TRY(load_V0(ctx, V0, V0_where, is_complex, seed));
  return start(ctx);
}

gplhr_status gplhr_iterate(gplhr_ctx* ctx, int32_t niter, gplhr_info* info) {
  if (!ctx) return GPLHR_EINVAL;
  if (!ctx->started) {
    ctx->err = "gplhr_iterate before gplhr_start";
    return GPLHR_EINVAL;
  }
  bool conv = false;
  return run_iterations(ctx, niter, info, &conv);
}

gplhr_status gplhr_solve(gplhr_ctx* ctx, const void* V0, int32_t V0_where, int32_t is_complex, uint64_t seed,
                         gplhr_info* info) {
  if (!ctx) return GPLHR_EINVAL;
  TRY(gplhr_start(ctx, V0, V0_where, is_complex, seed));
  bool conv = false;
  TRY(run_iterations(ctx, ctx->maxit, info, &conv));
  if (!conv) {
    ctx->err = "maxit reached before all pairs met tol";
    return GPLHR_ENOTCONV;
  }
  return GPLHR_OK;
}

namespace {
// x_j = V z_j / ||V z_j|| (FP64) into ctx->Tw3 (n x k, ld = k); returns Ze normalised.
gplhr_status eigvec_block(gplhr_ctx* ctx, SqMat* Ze_out) {
  const int k = ctx->k;
  SqMat Ze = gplhr::tri_eigvecs(ctx->RA, ctx->RB);
  for (int j = 0; j < k; ++j) {
    double zn = 0.0;
    for (int i = 0; i < k; ++i) zn += std::norm(Ze(i, j));
    zn = std::sqrt(zn);
    for (int i = 0; i < k; ++i) Ze(i, j) /= zn;
  }
  double2* hz = ctx->h_small;
  pack(hz, Ze, 0, k, 0, k);
  TRY(upload(ctx, ctx->dC1, hz, k * k));
  const Blk none{nullptr, 0};
  TRY(combine(ctx, {In{blkZ(ctx, 0), k, ctx->dC1, kOne}}, Blk{ctx->Tw3, k}, k, false, nullptr, none, -1, -1, true,
              0));
  if (Ze_out) *Ze_out = Ze;
  return GPLHR_OK;
}
}  // namespace

// GPLHR-EIG results: the Rayleigh-quotient pairs, X, the residuals of the last refresh;
// the Schur-form outputs (V, Q, RA, RB) are zero-filled (the variant keeps no Schur form).
gplhr_status eig_vectors(gplhr_ctx* ctx, double* alpha, double* beta, double* lambda, void* X, void* V, void* Q,
                         void* RA, void* RB, double* resid, int32_t where) {
  const int n = ctx->n, k = ctx->k;
  for (int j = 0; j < k; ++j) {
    const cd a = ctx->ea[j], b = ctx->eb[j];
    if (alpha) { alpha[2 * j] = a.real(); alpha[2 * j + 1] = a.imag(); }
    if (beta) { beta[2 * j] = b.real(); beta[2 * j + 1] = b.imag(); }
    if (lambda) {
      const cd l = std::abs(b) > 0 ? a / b : cd(INFINITY, 0.0);
      lambda[2 * j] = l.real();
      lambda[2 * j + 1] = l.imag();
    }
    if (resid) resid[j] = ctx->resid[j];
  }
  const size_t bytes = (size_t)n * k * sizeof(double2), rbytes = (size_t)k * k * sizeof(double2);
  if (X)
    CK(cudaMemcpyAsync(X, ctx->eX, bytes, where == GPLHR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       ctx->stream));
  void* outs[4] = {V, Q, RA, RB};
  const size_t sizes[4] = {bytes, bytes, rbytes, rbytes};
  for (int i = 0; i < 4; ++i)
    if (outs[i]) {
      if (where == GPLHR_DEVICE)
        CK(cudaMemsetAsync(outs[i], 0, sizes[i], ctx->stream));
      else
        std::memset(outs[i], 0, sizes[i]);
    }
  CK(cudaStreamSynchronize(ctx->stream));
  return GPLHR_OK;
}

gplhr_status gplhr_vectors(gplhr_ctx* ctx, double* alpha, double* beta, double* lambda, void* X, void* V,
                           void* Q, void* RA, void* RB, double* resid, int32_t where) {
  if (!ctx) return GPLHR_EINVAL;
  if (!ctx->started) {
    ctx->err = "gplhr_vectors before gplhr_start";
    return GPLHR_EINVAL;
  }
  if (ctx->eig) return eig_vectors(ctx, alpha, beta, lambda, X, V, Q, RA, RB, resid, where);
  const int n = ctx->n, k = ctx->k;
  const cudaMemcpyKind d2x = where == GPLHR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  for (int j = 0; j < k; ++j) {
    const cd a = ctx->RA(j, j), b = ctx->RB(j, j);
    if (alpha) { alpha[2 * j] = a.real(); alpha[2 * j + 1] = a.imag(); }
    if (beta) { beta[2 * j] = b.real(); beta[2 * j + 1] = b.imag(); }
    if (lambda) {
      const cd l = std::abs(b) > 0 ? a / b : cd(INFINITY, 0.0);
      lambda[2 * j] = l.real();
      lambda[2 * j + 1] = l.imag();
    }
  }
  // V, Q: the first k columns of Z, U (row stride s_max).  To the host they are packed into
  // a contiguous scratch block first (a strided copy of n rows of 16 k bytes each to
  // pageable memory is slow), then copied in one piece; the scratch is stream-ordered
  // against the copies.
  const struct {
    void* dst;
    const double2* src;
  } outs[2] = {{V, ctx->Z}, {Q, ctx->U}};
  for (const auto& o : outs) {
    if (!o.dst) continue;
    if (where == GPLHR_DEVICE) {
      CK(cudaMemcpy2DAsync(o.dst, k * sizeof(double2), o.src, ctx->s_max * sizeof(double2), k * sizeof(double2), n,
                           d2x, ctx->stream));
    } else {
      gplhr::copy_block_kernel<<<grid_for((size_t)n * k, 256, 8 * ctx->num_sms), 256, 0, ctx->stream>>>(
          n, k, o.src, ctx->s_max, ctx->Tw1, k);
      CK(cudaGetLastError());
      CK(cudaMemcpyAsync(o.dst, ctx->Tw1, (size_t)n * k * sizeof(double2), d2x, ctx->stream));
    }
  }
  SqMat Rout = ctx->RA, RBout = ctx->RB;
  if (!ctx->hasB) {  // B = I: R = M_A M_B^{-1} (A V M_B = V M_A, Eq. gschur2), RB = I
    SqMat Minv = SqMat::eye(k);
    // solve M_B^T-free: Rout = MA * inv(MB), MB upper triangular
    for (int c = 0; c < k; ++c)
      for (int i = k - 1; i >= 0; --i) {
        cd acc = (i == c) ? cd(1.0) : cd(0.0);
        for (int t = i + 1; t < k; ++t) acc -= ctx->MB(i, t) * Minv(t, c);
        Minv(i, c) = acc / ctx->MB(i, i);
      }
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) {
        cd acc = 0.0;
        for (int t = 0; t < k; ++t) acc += ctx->MA(i, t) * Minv(t, j);
        Rout(i, j) = acc;
      }
    RBout = SqMat::eye(k);
  }
  std::vector<double2> hr(k * k);
  if (RA) {
    pack(hr.data(), Rout, 0, k, 0, k);
    CK(cudaMemcpyAsync(RA, hr.data(), k * k * sizeof(double2),
                       where == GPLHR_DEVICE ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  if (RB) {
    pack(hr.data(), RBout, 0, k, 0, k);
    CK(cudaMemcpyAsync(RB, hr.data(), k * k * sizeof(double2),
                       where == GPLHR_DEVICE ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  if (X || resid) {
    // x_j = V z_j / ||V z_j||; fresh products A X, B X for the residuals
    SqMat Ze = gplhr::tri_eigvecs(ctx->RA, ctx->RB);
    for (int j = 0; j < k; ++j) {
      double zn = 0.0;
      for (int i = 0; i < k; ++i) zn += std::norm(Ze(i, j));
      zn = std::sqrt(zn);
      for (int i = 0; i < k; ++i) Ze(i, j) /= zn;
    }
    double2* hz = ctx->h_small;
    pack(hz, Ze, 0, k, 0, k);
    TRY(upload(ctx, ctx->dC1, hz, k * k));
    // scratch only: Rw carries the residual into the next gplhr_iterate
    Blk Xb{ctx->Tw3, k};
    const Blk none{nullptr, 0};
    TRY(combine(ctx, {In{blkZ(ctx, 0), k, ctx->dC1, kOne}}, Xb, k, false, nullptr, none, -1, -1, true, 0));
    if (resid) {
      Blk AX{ctx->Tw1, k}, BX{ctx->hasB ? ctx->Tw2 : ctx->Tw3, k};
      TRY(pair_products(ctx, Xb, k, AX, BX, false));
      double2* hb = ctx->h_small + k * k;
      double2* ha = ctx->h_small + 2 * k * k;
      for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) {
          hb[i * k + j] = i == j ? d2(ctx->RB(j, j)) : make_double2(0.0, 0.0);
          ha[i * k + j] = i == j ? d2(ctx->RA(j, j)) : make_double2(0.0, 0.0);
        }
      TRY(upload(ctx, ctx->dC2, hb, 2 * k * k));
      TRY(combine(ctx, {In{AX, k, ctx->dC2, kOne}, In{BX, k, ctx->dC2 + k * k, kMinusOne}}, none, k, false,
                  nullptr, none, 0, 0, true, 0));
      std::vector<double> nrm(k);
      CK(cudaMemcpyAsync(nrm.data(), ctx->d_norms, k * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
      for (int j = 0; j < k; ++j) {
        const double a = std::abs(ctx->RA(j, j)), b = std::abs(ctx->RB(j, j));
        resid[j] = std::sqrt(nrm[j]) / (b * ctx->normA + a * ctx->normB);
      }
    }
    if (X) CK(cudaMemcpyAsync(X, ctx->Tw3, (size_t)n * k * sizeof(double2), d2x, ctx->stream));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return GPLHR_OK;
}

void gplhr_destroy(gplhr_ctx* ctx) {
  if (!ctx) return;
  for (auto& g : ctx->seg_graphs) cudaGraphExecDestroy(g.second.exec);
  ctx->seg_graphs.clear();
  free_all(ctx);
  delete ctx;
}

const char* gplhr_last_error(const gplhr_ctx* ctx) {
  if (!ctx) return g_create_error.c_str();
  return ctx->err.c_str();
}

gplhr_status gplhr_spmm(gplhr_ctx* ctx, const void* X, int32_t ldx, int32_t w, void* AX, int32_t ldax, void* BX,
                        int32_t ldbx) {
  if (!ctx || !valid_block(X, ldx, w) || !valid_block(AX, ldax, w) || (ctx->hasB && BX && ldbx < w))
    return GPLHR_EINVAL;
  const bool withB = ctx->hasB && BX;
  TRY(launch_spmm_one(ctx, ctx->A, withB ? &ctx->B : nullptr, Blk{(double2*)X, ldx}, w, Blk{(double2*)AX, ldax},
                      Blk{(double2*)BX, ldbx}));
  CK(cudaStreamSynchronize(ctx->stream));
  return GPLHR_OK;
}

gplhr_status gplhr_precond_apply(gplhr_ctx* ctx, const void* X, int32_t ldx, int32_t w, void* Y, int32_t ldy) {
  if (!ctx || !valid_block(X, ldx, w) || !valid_block(Y, ldy, w) || w > ctx->k) return GPLHR_EINVAL;
  TRY(precond_apply(ctx, Blk{(double2*)X, ldx}, w, Blk{(double2*)Y, ldy}));
  CK(cudaStreamSynchronize(ctx->stream));
  return GPLHR_OK;
}

gplhr_status gplhr_gram(gplhr_ctx* ctx, const void* X, int32_t ldx, int32_t wx, const void* Y, int32_t ldy,
                        int32_t wy, void* C, int32_t arith) {
  if (!ctx || !valid_block(X, ldx, wx) || !valid_block(Y, ldy, wy) || !C || wx > std::max(ctx->s_max, 128) ||
      wy > 2 * ctx->s_max || arith < 0 || arith > 3)
    return GPLHR_EINVAL;
  const bool saved = ctx->bulk32;
  if (arith == 3) ctx->bulk32 = false;  // the FP64 product, on the tensor cores where the shape allows
  const gplhr_status st = gram(ctx, Blk{(double2*)X, ldx}, wx, Blk{(double2*)Y, ldy}, wy, Blk{nullptr, 0}, 0,
                               (double2*)C, nullptr, false, true, false, arith == 3 ? -1 : arith);
  ctx->bulk32 = saved;
  TRY(st);
  CK(cudaStreamSynchronize(ctx->stream));
  return GPLHR_OK;
}

gplhr_status gplhr_combine(gplhr_ctx* ctx, const void* X, int32_t ldx, int32_t w, const void* C, int32_t c,
                           void* Y, int32_t ldy, int32_t beta, int32_t arith) {
  if (!ctx || !valid_block(X, ldx, w) || !valid_block(Y, ldy, c) || !C || w < 1 || c < 1 || w > 2 * ctx->s_max ||
      c > 2 * ctx->s_max || arith < 0 || arith > 1 || beta < 0 || beta > 1 ||
      (X == Y && (c != w || ldy != ldx || beta != 0)))
    return GPLHR_EINVAL;
  CK(cudaMemsetAsync(ctx->d_diag + 2, 0, sizeof(int), ctx->stream));  // this call's time-out flag
  const bool tc = ctx->tc;
  ctx->tc = tc && arith == GPLHR_COMBINE_AUTO;
  const gplhr_status st = combine(ctx, {In{Blk{(double2*)X, ldx}, w, (const double2*)C, kOne}},
                                  Blk{(double2*)Y, ldy}, c, beta != 0, nullptr, Blk{nullptr, 0}, -1, -1, true, 0);
  ctx->tc = tc;
  TRY(st);
  CK(cudaMemcpyAsync(ctx->h_diag, ctx->d_diag, 3 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (ctx->h_diag[2] != 0) {
    ctx->err = "tensor-core product: wait for completion gave up";
    return GPLHR_ETIMEOUT;
  }
  return GPLHR_OK;
}

gplhr_status gplhr_spmm_shape(gplhr_ctx* ctx, int32_t w, int32_t fp32, int32_t* threads, int32_t* grid_per_sm,
                              double* us, double* us_default) {
  if (!ctx || w < 1 || w > 32 * (fp32 ? 2 : 1)) return GPLHR_EINVAL;
  const int V = fp32 ? 2 : 1;
  int G = 4;
  while (G * V < w) G <<= 1;
  gplhr_ctx::SpmmShape sh;
  const auto it = ctx->spmm_shape.find(4 * G + V);
  if (it != ctx->spmm_shape.end()) sh = it->second;
  if (threads) *threads = sh.threads;
  if (grid_per_sm) *grid_per_sm = sh.gridmul;
  if (us) *us = sh.us;
  if (us_default) *us_default = sh.us_default;
  return GPLHR_OK;
}

gplhr_status gplhr_set_deflation(gplhr_ctx* ctx, const void* V1, const void* Q1, int32_t k1, int32_t where) {
  if (!ctx) return GPLHR_EINVAL;
  if (k1 < 0 || k1 > 256 || (k1 > 0 && (!V1 || (ctx->hasB && !Q1))) || (where != GPLHR_HOST && where != GPLHR_DEVICE) ||
      (int64_t)k1 + ctx->s_max > ctx->n || (size_t)k1 * ctx->k > (size_t)2 * ctx->s_max * ctx->s_max) {
    ctx->err = "gplhr_set_deflation: need 0 <= k1 <= 256, k1 + (m+3)k <= n, k1 k <= 2 ((m+3)k)^2, V1 (and Q1 "
               "when B != I) given, where HOST or DEVICE";
    return GPLHR_EINVAL;
  }
  if ((ctx->gm_steps > 0 || ctx->eig) && k1 > 0) {
    ctx->err = "gplhr_set_deflation: not available with inner GMRES steps or the eigenvector variant";
    return GPLHR_EINVAL;
  }
  CK(cudaStreamSynchronize(ctx->stream));
  for (auto& g : ctx->seg_graphs) cudaGraphExecDestroy(g.second.exec);  // launch sequences change
  ctx->seg_graphs.clear();
  if (ctx->dV1) cudaFree(ctx->dV1);
  if (ctx->dQ1) cudaFree(ctx->dQ1);
  ctx->dV1 = ctx->dQ1 = nullptr;
  ctx->k1 = 0;
  if (k1 == 0) return GPLHR_OK;
  const size_t bytes = (size_t)ctx->n * k1 * sizeof(double2);
  const cudaMemcpyKind kind = where == GPLHR_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  CK(cudaMalloc(&ctx->dV1, bytes));
  CK(cudaMemcpyAsync(ctx->dV1, V1, bytes, kind, ctx->stream));
  if (ctx->hasB) {
    CK(cudaMalloc(&ctx->dQ1, bytes));
    CK(cudaMemcpyAsync(ctx->dQ1, Q1, bytes, kind, ctx->stream));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->k1 = k1;
  return GPLHR_OK;
}

gplhr_status gplhr_orth(gplhr_ctx* ctx, void* X, int32_t ldx, int32_t w, void* Rinv) {
  if (!ctx || !valid_block(X, ldx, w) || w > ctx->s_max) return GPLHR_EINVAL;
  TRY(orth_against(ctx, Blk{nullptr, 0}, 0, Blk{(double2*)X, ldx}, w));
  if (Rinv) {
    // R^{-1} of the whole orth = Rinv_0 Rinv_1 (Rinv_2): accumulate on the host
    const int smax2 = ctx->s_max * ctx->s_max;
    std::vector<double2> h(3 * (size_t)smax2);
    CK(cudaMemcpyAsync(h.data(), ctx->dRinv, 3 * smax2 * sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    SqMat acc = SqMat::eye(w);
    for (int p = 0; p < 3; ++p) {
      SqMat Rp(w), t(w);
      for (int i = 0; i < w; ++i)
        for (int j = 0; j < w; ++j) Rp(i, j) = cd(h[p * smax2 + i * w + j].x, h[p * smax2 + i * w + j].y);
      for (int i = 0; i < w; ++i)
        for (int j = 0; j < w; ++j) {
          cd s = 0.0;
          for (int l = 0; l < w; ++l) s += acc(i, l) * Rp(l, j);
          t(i, j) = s;
        }
      acc = t;
    }
    std::vector<double2> o(w * w);
    pack(o.data(), acc, 0, w, 0, w);
    CK(cudaMemcpy(Rinv, o.data(), w * w * sizeof(double2), cudaMemcpyHostToDevice));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return GPLHR_OK;
}

gplhr_status gplhr_profile(gplhr_ctx* ctx, int32_t enable) {
  if (!ctx) return GPLHR_EINVAL;
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->prof_on = enable != 0;
  ctx->ev_rec.clear();
  for (int c = 0; c < 8; ++c) {
    ctx->k_flops[c] = ctx->k_bytes[c] = 0.0;
    ctx->k_launch[c] = 0;
  }
  ctx->n_launch = 0;
  return GPLHR_OK;
}

gplhr_status gplhr_profile_read(gplhr_ctx* ctx, int32_t kclass, double* ms, int64_t* launches, double* flops,
                                double* bytes) {
  if (!ctx || kclass < 0 || kclass >= KC_N) return GPLHR_EINVAL;
  CK(cudaStreamSynchronize(ctx->stream));
  double t = 0.0;
  for (const auto& r : ctx->ev_rec) {
    if (r.first != kclass) continue;
    float e = 0.f;
    CK(cudaEventElapsedTime(&e, ctx->ev_pool[r.second], ctx->ev_pool[r.second + 1]));
    t += e;
  }
  if (ms) *ms = t;
  if (launches) *launches = ctx->k_launch[kclass];
  if (flops) *flops = ctx->k_flops[kclass];
  if (bytes) *bytes = ctx->k_bytes[kclass];
  return GPLHR_OK;
}

gplhr_status gplhr_gram_noalloc(int64_t n, const void* X, int32_t ldx, int32_t wx, const void* Y, int32_t ldy,
                                int32_t wy, void* C, void* stream) {
  // n <= 2^30: the kernels index rows in int, and the last chunk's end r0 + rows as well
  // as its last 16-row step stay below 2^31 with that margin
  if (n < 1 || n > kNoallocMaxRows || wx < 1 || wy < 1 || ldx < wx || ldy < wy || !X || !Y || !C) {
    g_create_error = "gplhr_gram_noalloc: need 1 <= n <= 2^30, w >= 1, ld >= w, non-null pointers";
    return GPLHR_EINVAL;
  }
  if ((int64_t)wx * wy > kNoallocMaxOut || wx + wy > kNoallocMaxCols) {
    g_create_error = "gplhr_gram_noalloc: wx * wy must be <= 16384 and wx + wy <= 768 (fixed scratch size)";
    return GPLHR_EINVAL;
  }
  double2* scratch = nullptr;
  int nsm = 0;
  gplhr_status st = noalloc_setup(&scratch, &nsm);
  if (st != GPLHR_OK) return st;
  const int nn = (int)n;
  const int nout = wx * wy;
  const int64_t R = gplhr::GRAM_ROWS;
  int acc = 8;
  while (acc > 1 && (nout + acc - 1) / acc < 128) acc >>= 1;
  const int groups = (nout + acc - 1) / acc;
  const int G = std::min(groups, gplhr::GRAM_THREADS);
  const int RG = gplhr::GRAM_THREADS / G;
  const int ntile = (groups + G - 1) / G;
  // row chunks (one partial sum each) in 64-bit arithmetic: at most 4 CTAs per SM, one
  // 16-row step per chunk at least, and no more partial sums than the scratch holds
  int64_t nch = std::max<int64_t>(1, (4 * (int64_t)std::max(nsm, 1)) / ntile);
  nch = std::min<int64_t>(nch, std::max<int64_t>(1, (n + R - 1) / R));
  nch = std::min<int64_t>(nch, (int64_t)(kNoallocScratchElems / nout));
  int64_t rows64 = (n + nch - 1) / nch;
  rows64 = ((rows64 + R - 1) / R) * R;
  const int nchunk = (int)((n + rows64 - 1) / rows64);
  const int rows = (int)rows64;
  const dim3 grid(nchunk, ntile);
  const size_t smem =
      std::max((size_t)gplhr::GRAM_ROWS * (wx + wy), (size_t)RG * G * acc) * sizeof(double2);
  cudaStream_t strm = (cudaStream_t)stream;
  const double2* Xp = (const double2*)X;
  const double2* Yp = (const double2*)Y;
  const double2* none = nullptr;
  switch (acc) {
    case 8:
      gplhr::gram_partial_kernel<8><<<grid, gplhr::GRAM_THREADS, smem, strm>>>(
          nn, rows, Xp, ldx, wx, Yp, ldy, wy, none, 0, 0, 0, nout, G, RG, scratch, nullptr);
      break;
    case 4:
      gplhr::gram_partial_kernel<4><<<grid, gplhr::GRAM_THREADS, smem, strm>>>(
          nn, rows, Xp, ldx, wx, Yp, ldy, wy, none, 0, 0, 0, nout, G, RG, scratch, nullptr);
      break;
    case 2:
      gplhr::gram_partial_kernel<2><<<grid, gplhr::GRAM_THREADS, smem, strm>>>(
          nn, rows, Xp, ldx, wx, Yp, ldy, wy, none, 0, 0, 0, nout, G, RG, scratch, nullptr);
      break;
    default:
      gplhr::gram_partial_kernel<1><<<grid, gplhr::GRAM_THREADS, smem, strm>>>(
          nn, rows, Xp, ldx, wx, Yp, ldy, wy, none, 0, 0, 0, nout, G, RG, scratch, nullptr);
      break;
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    gplhr::gram_reduce_kernel<<<(nout + gplhr::GRED_WARPS - 1) / gplhr::GRED_WARPS, 32 * gplhr::GRED_WARPS, 0,
                                 strm>>>(nchunk, nout, wx, wy, 0, scratch, (double2*)C, wy, nullptr);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    g_create_error = std::string("gplhr_gram_noalloc: launch: ") + cudaGetErrorString(e);
    return GPLHR_ECUDA;
  }
  return GPLHR_OK;
}

gplhr_status gplhr_grad(gplhr_ctx* right, gplhr_ctx* left, const double* G, void* dA_vals, void* dB_vals,
                        int32_t where) {
  if (!right || !left || !G || (!dA_vals && !dB_vals)) {
    g_create_error = "gplhr_grad: contexts, G and at least one output are required";
    return GPLHR_EINVAL;
  }
  gplhr_ctx* ctx = right;
  if (!right->started || !left->started || right->eig || left->eig || right->n != left->n || right->k != left->k ||
      right->hasB != left->hasB || (dB_vals && !right->hasB)) {
    ctx->err = "gplhr_grad: both contexts must be solved, with equal n, k and B kind (dB needs B != I)";
    return GPLHR_EINVAL;
  }
  const int n = ctx->n, k = ctx->k;
  // pair right lambda_i with the left eigenvalue mu_j ~ conj(lambda_i)
  std::vector<cd> lam(k), mu(k);
  for (int j = 0; j < k; ++j) {
    lam[j] = right->RA(j, j) / right->RB(j, j);
    mu[j] = left->RA(j, j) / left->RB(j, j);
  }
  std::vector<int> perm(k, -1);
  for (int i = 0; i < k; ++i) {
    int best = -1, nmatch = 0;
    double bd = 1e300;
    const double tol = 1e-6 * std::max(std::abs(lam[i]), 1e-300);
    for (int j = 0; j < k; ++j) {
      const double d = std::abs(std::conj(mu[j]) - lam[i]);
      if (d <= tol) ++nmatch;
      if (d < bd) { bd = d; best = j; }
    }
    if (bd > tol || nmatch != 1) {
      ctx->err = "gplhr_grad: no unique left eigenvalue matches lambda_" + std::to_string(i);
      return GPLHR_EINVAL;
    }
    perm[i] = best;
  }
  // right vectors X (right->Tw3), left vectors Y (left->Tw3), Y permuted into right->Tw2
  TRY(eigvec_block(left, nullptr));
  CK(cudaStreamSynchronize(left->stream));
  TRY(eigvec_block(right, nullptr));
  {
    double2* hp = ctx->h_small + k * k;
    for (int i = 0; i < k * k; ++i) hp[i] = make_double2(0.0, 0.0);
    for (int i = 0; i < k; ++i) hp[perm[i] * k + i] = make_double2(1.0, 0.0);
    TRY(upload(ctx, ctx->dC2, hp, k * k));
    const Blk none{nullptr, 0};
    TRY(combine(ctx, {In{Blk{left->Tw3, k}, k, ctx->dC2, kOne}}, Blk{ctx->Tw2, k}, k, false, nullptr, none, -1, -1,
                true, 0));
  }
  const Blk X{ctx->Tw3, k}, Y{ctx->Tw2, k};
  // d_i = y_i^* B x_i
  Blk BX = X;
  if (ctx->hasB) {
    BX = Blk{ctx->Tw1, k};
    TRY(launch_spmm_one(ctx, ctx->B, nullptr, X, k, BX, Blk{nullptr, 0}, false));
  }
  TRY(gram(ctx, Y, k, BX, k, Blk{nullptr, 0}, 0, ctx->dGram));
  std::vector<double2> D(k * k);
  CK(cudaMemcpyAsync(D.data(), ctx->dGram, k * k * sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  double2* hc = ctx->h_small + 2 * k * k;
  for (int i = 0; i < k; ++i) {
    const cd d(D[i * k + i].x, D[i * k + i].y);
    if (std::abs(d) == 0.0) {
      ctx->err = "gplhr_grad: y_i^* B x_i = 0 (defective or badly paired eigenvalue)";
      return GPLHR_ENUMERIC;
    }
    const cd a = cd(G[2 * i], G[2 * i + 1]) / std::conj(d);
    hc[i] = d2(a);
    hc[k + i] = d2(-std::conj(lam[i]) * a);
  }
  TRY(upload(ctx, ctx->dC1, hc, 2 * k));
  auto scatter = [&](const DevCsr& M, const double2* coef, void* outp) -> gplhr_status {
    const bool cplx = M.dtype == GPLHR_C128;
    const size_t bytes = (size_t)M.nnz * (cplx ? 16 : 8);
    void* dst = outp;
    void* tmp = nullptr;
    if (where != GPLHR_DEVICE) {
      CK(cudaMalloc(&tmp, std::max<size_t>(bytes, 16)));
      dst = tmp;
    }
    const int grid = grid_for((size_t)n, 8, ctx->num_sms * 16);
    if (cplx)
      gplhr::adjoint_scatter_kernel<double2><<<grid, 256, 0, ctx->stream>>>(n, M.rowptr, M.col, Y.p, Y.ld, X.p, X.ld,
                                                                           k, coef, (double2*)dst);
    else
      gplhr::adjoint_scatter_kernel<double><<<grid, 256, 0, ctx->stream>>>(n, M.rowptr, M.col, Y.p, Y.ld, X.p, X.ld,
                                                                          k, coef, (double*)dst);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && tmp) {
      e = cudaMemcpyAsync(outp, tmp, bytes, cudaMemcpyDeviceToHost, ctx->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    }
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess) {
      ctx->err = std::string("gplhr_grad: ") + cudaGetErrorString(e);
      return GPLHR_ECUDA;
    }
    return GPLHR_OK;
  };
  if (dA_vals) TRY(scatter(ctx->A, ctx->dC1, dA_vals));
  if (dB_vals) TRY(scatter(ctx->B, ctx->dC1 + k, dB_vals));
  CK(cudaStreamSynchronize(ctx->stream));
  return GPLHR_OK;
}

// Batched driver: contexts are independent (own streams and buffers); a pool of host
// threads takes them one at a time, so the host QZ and synchronisation of one pencil
// overlap the device work of the others.
static gplhr_status run_batched(int32_t nctx, gplhr_ctx* const* ctxs, int32_t nthreads, gplhr_status* statuses,
                                const std::function<gplhr_status(int)>& job) {
  if (nctx < 0 || (nctx > 0 && !ctxs)) return GPLHR_EINVAL;
  for (int i = 0; i < nctx; ++i)
    if (!ctxs[i]) return GPLHR_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GPLHR_ECUDA;
  const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
  const int nt = std::max(1, std::min<int>(nthreads > 0 ? nthreads : hw, nctx));
  std::vector<gplhr_status> st(nctx, GPLHR_OK);
  std::atomic<int> next(0);
  auto worker = [&]() {
    cudaSetDevice(dev);
    for (int i = next.fetch_add(1); i < nctx; i = next.fetch_add(1)) st[i] = job(i);
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < nt; ++t) pool.emplace_back(worker);
  worker();
  for (auto& th : pool) th.join();
  gplhr_status first = GPLHR_OK;
  for (int i = 0; i < nctx; ++i) {
    if (statuses) statuses[i] = st[i];
    if (first == GPLHR_OK && st[i] != GPLHR_OK) first = st[i];
  }
  return first;
}

gplhr_status gplhr_iterate_batched(int32_t nctx, gplhr_ctx* const* ctxs, int32_t niter, gplhr_info* infos,
                                   gplhr_status* statuses, int32_t nthreads) {
  return run_batched(nctx, ctxs, nthreads, statuses, [&](int i) {
    return gplhr_iterate(ctxs[i], niter, infos ? infos + i : nullptr);
  });
}

gplhr_status gplhr_create_batched(int32_t nctx, const gplhr_csr* const* A, const gplhr_csr* const* B,
                                  const double* sigma, const int32_t* k, const int32_t* m,
                                  const gplhr_precond* const* T, const gplhr_opts* const* opts, gplhr_ctx** out,
                                  gplhr_status* statuses, int32_t nthreads) {
  if (nctx < 0 || (nctx > 0 && (!A || !sigma || !k || !m || !out))) {
    g_create_error = "gplhr_create_batched: need nctx >= 0 and non-null A, sigma, k, m, out";
    return GPLHR_EINVAL;
  }
  for (int i = 0; i < nctx; ++i) out[i] = nullptr;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    g_create_error = "gplhr_create_batched: no CUDA device";
    return GPLHR_ECUDA;
  }
  std::vector<gplhr_status> st(nctx, GPLHR_OK);
  std::vector<std::string> msg(nctx);
  std::atomic<int> next(0);
  auto worker = [&]() {
    cudaSetDevice(dev);
    for (int i = next.fetch_add(1); i < nctx; i = next.fetch_add(1)) {
      st[i] = gplhr_create(A[i], B ? B[i] : nullptr, sigma[2 * i], sigma[2 * i + 1], k[i], m[i], T ? T[i] : nullptr,
                           opts ? opts[i] : nullptr, &out[i]);
      if (st[i] != GPLHR_OK) msg[i] = g_create_error;  // this worker thread's message
    }
  };
  const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
  const int nt = std::max(1, std::min<int>(nthreads > 0 ? nthreads : hw, nctx));
  std::vector<std::thread> pool;
  for (int t = 1; t < nt; ++t) pool.emplace_back(worker);
  worker();
  for (auto& th : pool) th.join();
  gplhr_status first = GPLHR_OK;
  int bad = -1;
  for (int i = 0; i < nctx; ++i) {
    if (statuses) statuses[i] = st[i];
    if (first == GPLHR_OK && st[i] != GPLHR_OK) {
      first = st[i];
      bad = i;
    }
  }
  if (first != GPLHR_OK) {  // all or nothing: the contexts that were created are freed
    for (int i = 0; i < nctx; ++i) {
      gplhr_destroy(out[i]);
      out[i] = nullptr;
    }
    g_create_error = "gplhr_create_batched: context " + std::to_string(bad) + ": " + msg[bad];
  }
  return first;
}

gplhr_status gplhr_solve_batched(int32_t nctx, gplhr_ctx* const* ctxs, const void* const* V0,
                                 const int32_t* V0_where, const int32_t* is_complex, const uint64_t* seeds,
                                 gplhr_info* infos, gplhr_status* statuses, int32_t nthreads) {
  return run_batched(nctx, ctxs, nthreads, statuses, [&](int i) {
    return gplhr_solve(ctxs[i], V0 ? V0[i] : nullptr, V0_where ? V0_where[i] : GPLHR_HOST,
                       is_complex ? is_complex[i] : 0, seeds ? seeds[i] : 0, infos ? infos + i : nullptr);
  });
}

// Persistent batched iteration (pk_iterate): checks shared by the two entry points.
static gplhr_status pk_check(int32_t nctx, gplhr_ctx* const* ctxs, bool need_started) {
  if (nctx < 0 || (nctx > 0 && !ctxs)) {
    g_create_error = "persistent batch: need nctx >= 0 and a context array";
    return GPLHR_EINVAL;
  }
  std::vector<const gplhr_ctx*> seen;
  for (int i = 0; i < nctx; ++i) {
    const gplhr_ctx* c = ctxs[i];
    const char* why = nullptr;
    if (!c) why = "null context";
    else if (std::find(seen.begin(), seen.end(), c) != seen.end()) why = "a context appears twice";
    else if (need_started && !c->started) why = "context not started (gplhr_start)";
    else if (c->eig) why = "GPLHR-EIG contexts are not supported";
    else if (c->gm_steps > 0) why = "inner GMRES preconditioning is not supported (its least squares runs on the host)";
    else if (c->prof_on) why = "profiling is on";
    if (why) {
      g_create_error = "persistent batch: context " + std::to_string(i) + ": " + why;
      return GPLHR_EINVAL;
    }
    seen.push_back(c);
  }
  return GPLHR_OK;
}

static gplhr_status pk_finish(int32_t nctx, gplhr_ctx* const* ctxs, const std::vector<gplhr_status>& st,
                              const std::vector<char>& conv, bool need_conv, gplhr_info* infos,
                              gplhr_status* statuses, const PkRunner& R, gplhr_persist_stats* stats) {
  gplhr_status first = GPLHR_OK;
  for (int i = 0; i < nctx; ++i) {
    gplhr_status si = st[i];
    if (si == GPLHR_OK && need_conv && !conv[i]) {
      ctxs[i]->err = "maxit reached before all pairs met tol";
      si = GPLHR_ENOTCONV;
    }
    fill_info(ctxs[i], infos ? infos + i : nullptr);
    if (statuses) statuses[i] = si;
    if (first == GPLHR_OK && si != GPLHR_OK) first = si;
  }
  if (stats) {
    stats->launches = R.launches;
    stats->steps = R.steps;
    stats->ops = R.ops;
    stats->grid = R.grid;
    stats->record_ms = R.record_ms;
    stats->build_ms = R.build_ms;
    stats->qz_ms = R.qz_ms;
    stats->wait_ms = R.wait_ms;
  }
  if (!R.err.empty()) g_create_error = R.err;
  return first;
}

gplhr_status gplhr_iterate_persistent(int32_t nctx, gplhr_ctx* const* ctxs, int32_t niter, gplhr_info* infos,
                                      gplhr_status* statuses, int32_t nthreads, gplhr_persist_stats* stats) {
  TRY(pk_check(nctx, ctxs, true));
  if (niter < 0) {
    g_create_error = "persistent batch: niter < 0";
    return GPLHR_EINVAL;
  }
  std::vector<int> cap(nctx);
  for (int i = 0; i < nctx; ++i) cap[i] = ctxs[i]->it + niter;
  const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
  PkRunner R;
  std::vector<gplhr_status> st;
  std::vector<char> conv;
  pk_iterate(nctx, ctxs, cap, nthreads > 0 ? nthreads : hw, st, conv, R);
  return pk_finish(nctx, ctxs, st, conv, false, infos, statuses, R, stats);
}

gplhr_status gplhr_solve_persistent(int32_t nctx, gplhr_ctx* const* ctxs, const void* const* V0,
                                    const int32_t* V0_where, const int32_t* is_complex, const uint64_t* seeds,
                                    gplhr_info* infos, gplhr_status* statuses, int32_t nthreads,
                                    gplhr_persist_stats* stats) {
  TRY(pk_check(nctx, ctxs, false));
  const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
  const int nt = nthreads > 0 ? nthreads : hw;
  // steps 1-4 of every context on its own stream (host threads), then the iterations
  std::vector<gplhr_status> st0(nctx, GPLHR_OK);
  run_batched(nctx, ctxs, nt, st0.data(), [&](int i) {
    return gplhr_start(ctxs[i], V0 ? V0[i] : nullptr, V0_where ? V0_where[i] : GPLHR_HOST,
                       is_complex ? is_complex[i] : 0, seeds ? seeds[i] : 0);
  });
  std::vector<gplhr_ctx*> ok;
  std::vector<int> where;
  for (int i = 0; i < nctx; ++i)
    if (st0[i] == GPLHR_OK) {
      ok.push_back(ctxs[i]);
      where.push_back(i);
    }
  std::vector<int> cap(ok.size());
  for (size_t j = 0; j < ok.size(); ++j) cap[j] = ok[j]->maxit;
  PkRunner R;
  std::vector<gplhr_status> st1;
  std::vector<char> conv1;
  pk_iterate((int)ok.size(), ok.data(), cap, nt, st1, conv1, R);
  std::vector<gplhr_status> st(nctx);
  std::vector<char> conv(nctx, 0);
  for (int i = 0; i < nctx; ++i) st[i] = st0[i];
  for (size_t j = 0; j < ok.size(); ++j) {
    st[where[j]] = st1[j];
    conv[where[j]] = conv1[j];
  }
  return pk_finish(nctx, ctxs, st, conv, true, infos, statuses, R, stats);
}

gplhr_status gplhr_ordqz(int32_t s, const double* Phi, const double* Psi, double sigma_re, double sigma_im,
                         double* RA, double* RB, double* YL, double* YR) {
  if (s < 0 || (s > 0 && (!Phi || !Psi || !RA || !RB || !YL || !YR))) return GPLHR_EINVAL;
  SqMat P(s), S(s), ra, rb, yl, yr;
  for (int i = 0; i < s * s; ++i) {
    P.a[i] = cd(Phi[2 * i], Phi[2 * i + 1]);
    S.a[i] = cd(Psi[2 * i], Psi[2 * i + 1]);
  }
  if (!gplhr::ordered_qz(P, S, cd(sigma_re, sigma_im), ra, rb, yl, yr)) return GPLHR_ENOTCONV;
  for (int i = 0; i < s * s; ++i) {
    RA[2 * i] = ra.a[i].real(); RA[2 * i + 1] = ra.a[i].imag();
    RB[2 * i] = rb.a[i].real(); RB[2 * i + 1] = rb.a[i].imag();
    YL[2 * i] = yl.a[i].real(); YL[2 * i + 1] = yl.a[i].imag();
    YR[2 * i] = yr.a[i].real(); YR[2 * i + 1] = yr.a[i].imag();
  }
  return GPLHR_OK;
}

gplhr_status gplhr_ordqz_device(int32_t s, const void* Phi, const void* Psi, double sigma_re, double sigma_im,
                                int32_t nsort, void* RA, void* RB, void* YL, void* YR, int32_t* status, void* stream) {
  if (s < 1 || s > gplhr::DQZ_SMAX || !Phi || !Psi || !RA || !RB || !YL || !YR || !status) {
    g_create_error = "gplhr_ordqz_device: need 1 <= s <= 80 and device pointers";
    return GPLHR_EINVAL;
  }
  cudaError_t e = cudaFuncSetAttribute(gplhr::ordqz_device_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)gplhr::dqz_smem_bytes(gplhr::DQZ_SMAX));
  if (e == cudaSuccess) {
    gplhr::ordqz_device_kernel<<<1, gplhr::DQZ_THREADS, gplhr::dqz_smem_bytes(s), (cudaStream_t)stream>>>(
        s, (const double2*)Phi, (const double2*)Psi, make_double2(sigma_re, sigma_im), nsort, (double2*)RA,
        (double2*)RB, (double2*)YL, (double2*)YR, status);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    g_create_error = std::string("gplhr_ordqz_device: ") + cudaGetErrorString(e);
    return GPLHR_ECUDA;
  }
  return GPLHR_OK;
}

gplhr_status gplhr_mfactors(int32_t k, const double* RA, const double* RB, double* MA, double* MB) {
  if (k < 0 || (k > 0 && (!RA || !RB || !MA || !MB))) return GPLHR_EINVAL;
  SqMat ra(k), rb(k), ma, mb;
  for (int i = 0; i < k * k; ++i) {
    ra.a[i] = cd(RA[2 * i], RA[2 * i + 1]);
    rb.a[i] = cd(RB[2 * i], RB[2 * i + 1]);
  }
  gplhr::m_factors(ra, rb, ma, mb);
  for (int i = 0; i < k * k; ++i) {
    MA[2 * i] = ma.a[i].real(); MA[2 * i + 1] = ma.a[i].imag();
    MB[2 * i] = mb.a[i].real(); MB[2 * i + 1] = mb.a[i].imag();
  }
  return GPLHR_OK;
}

}  // extern "C"
