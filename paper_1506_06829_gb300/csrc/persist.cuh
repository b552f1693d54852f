// Persistent kernel of the batched iteration: one launch runs a whole device segment of
// an iteration (Algorithm 2, steps 7-24, steps 25-28, or the residual with its column
// norms) for every context of a batch.
//
// The host records each context's segment as the list of launches it would make (kernel,
// grid, arguments), in program order.  A launch's CTAs become "virtual" CTAs (items) of
// the persistent kernel.  A launch is ready once its context's previous launch has
// finished all its items; the kernel's CTAs look for work among the contexts' current
// launches (one warp tests 32 contexts at once, in the host's priority order: the
// largest contexts, whose chains of launches are the longest, first), claim an item of
// a ready launch with an atomic counter, run the recorded kernel's body for it and count
// it finished.  The contexts thus advance independently and no CTA waits behind work
// that is not ready while other work is.
//
// Launched cooperatively (all CTAs resident).  A CTA that finds no ready work sleeps
// briefly and looks again; if nothing becomes ready within a time limit on the global
// timer the kernel records GPLHR_ETIMEOUT and every CTA returns.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "kernels.cuh"

namespace gplhr {

constexpr int PK_THREADS = 256;
// Resident CTAs per SM.  Most steps stream blocks from HBM through bodies written for
// full-GPU grids (stage a tile, synchronise, compute, store), so memory parallelism comes
// from resident warps: 4 CTAs (64 registers a thread, with some spills in the widest SpMM
// and Gram bodies) measured 20.6 ms per FP64 iteration of the 80-context batched workload
// against 22.9 ms with 3 CTAs and 23.1 ms with 2 (128 registers, no spills); 9.6 / 11.1 /
// 12.6 ms in mixed precision.
constexpr int PK_CTAS_PER_SM = 4;

enum PkKind : int {
  PK_BYTES = 1,   // PkBytes: plain device-to-device copy
  PK_AXPBY,       // PkAxpby
  PK_COPY_BLOCK,  // PkCopy
  PK_TO_C64,      // PkToC64
  PK_GRAM_REDUCE, // PkGramRed
  PK_NORM_REDUCE, // PkNormRed
  PK_CHOL,        // PkChol
  PK_COMBINE_D,   // PkComb, FP64
  PK_COMBINE_F,   // PkComb, FP32
  PK_JACOBI_D,    // PkJacobi
  PK_JACOBI_F,
  PK_BJ_DD,       // PkBj: FP64 arithmetic, complex128 inverse blocks
  PK_BJ_FD,       // FP32 arithmetic, complex128 blocks
  PK_BJ_FF,       // FP32 arithmetic, complex64 blocks
  PK_COPY_RAW,    // PkRaw: bytes between device and pinned host memory
  PK_GRAM_BASE = 32,  // + 4 mode + log2(ACC): mode 0 FP64, 1 FP32, 2 exact products (PkGram)
  PK_SPMM_BASE = 64,  // + spmm_code(): PkSpmm
  PK_KIND_END = 96
};

// SpMM kind: FP32 (T = float, V = 2) or FP64, A and B real or complex, G = 4 << gi.
__host__ __device__ constexpr int pk_spmm_code(int fp32, int acplx, int bcplx, int gi) {
  return PK_SPMM_BASE + (fp32 | (acplx << 1) | (bcplx << 2) | (gi << 3));
}

struct PkBytes {
  const double2* src;
  double2* dst;
  int64_t count;  // double2 elements
};
struct PkRaw {
  const unsigned char* src;
  unsigned char* dst;
  int64_t bytes;
};
struct PkAxpby {
  int n, w, ld1, ld2, ldy;
  double2 alpha, beta;
  const double2* X1;
  const double2* X2;
  double2* Y;
};
struct PkCopy {
  int n, w, ldx, ldy;
  const double2* X;
  double2* Y;
};
struct PkToC64 {
  int n, w, ldx, ldy;
  const double2* X;
  float2* Y;
};
struct PkGramRed {
  int nchunk, nout, wx, wy, herm, ldc;
  const double2* partial;
  double2* C;
  const int* skip;
};
struct PkNormRed {
  int nb, nc;
  const double* part;
  double* out;
};
struct PkChol {
  int w;
  int64_t n;
  const double2* G;
  double2* Rinv;
  int* status;
  const int* skip;
  int* fallback;
  double2* Rout;
  double2* work;  // null: shared memory; else 2 w^2 values of global memory
};
// Dynamic shared memory above which a Cholesky runs on global work memory instead, so
// that wide blocks (32 w^2 bytes: 131 KB at w = 64) do not cut the kernel's residency.
constexpr size_t PK_CHOL_SMEM_MAX = 48 * 1024;
struct PkComb {
  int n, rows_per_cta;
  CombArgs a;
};
struct PkJacobi {
  int n, w, ldx, ldy;
  const double2* d;
  const double2* X;
  double2* Y;
};
struct PkBj {
  int n, bs, w, ldx, ldy, bpc;
  const void* Tinv;
  const double2* X;
  double2* Y;
};
struct PkGram {
  int n, rows, ldx, wx, ldy0, wy0, ldy1, wy1, herm, nout, G, RG;
  const double2* X;
  const double2* Y0;
  const double2* Y1;
  double2* partial;
  const int* skip;
};
struct PkSpmm {
  int n, hasB, ldx, w, ldax, ldbx;
  const int* arp;
  const int* acol;
  const void* aval;
  const int* brp;
  const int* bcol;
  const void* bval;
  const void* X;
  double2* AX;
  double2* BX;
};

// One recorded launch: kind, virtual grid gx x gy, arguments at byte offset argoff of the
// argument pool (16-byte aligned).
struct PkOp {
  int kind, gx, gy;
  unsigned argoff;
};

// Device program, context-major: context c (in priority order) owns ops
// ctx_first[c] .. ctx_first[c] + ctx_nops[c] - 1 in program order; op o has vcount[o]
// items.  Zeroed before each launch: claimed[o] (items handed out), done[o] (items
// finished), cur[c] (the context's current op).
struct PkProgram {
  const PkOp* ops;
  const unsigned char* args;
  const int* vcount;
  const int* ctx_first;
  const int* ctx_nops;
  int* claimed;
  int* done;
  int* cur;
  int nops, nctx;
};

// Kernel state, zeroed by the host before each launch.
struct PkQueue {
  int abort;
  int pad[3];
};

__device__ __forceinline__ unsigned long long pk_globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int pk_ld(const int* p) { return *(volatile const int*)p; }

// Warp 0 of the CTA: claim an item of a ready op.  Lane l tests the contexts c = base + l
// (their current op: claimable items left, previous op finished; probe, a test hook,
// asks the previous op for one item more than it has, so nothing after a context's first
// op is ever ready); the lowest ready context (highest priority) is tried first.  Returns
// the op (>= 0, *item set), -1 if nothing is ready now, -2 if every context has finished.
__device__ __forceinline__ int pk_claim(const PkProgram& p, int probe, int* item) {
  const int lane = threadIdx.x & 31;
  bool all_finished = true;
  for (int base = 0; base < p.nctx; base += 32) {
    const int c = base + lane;
    int o = -1, j = 0;
    bool ready = false;
    if (c < p.nctx) {
      j = pk_ld(p.cur + c);
      if (j < p.ctx_nops[c]) {
        o = p.ctx_first[c] + j;
        ready = pk_ld(p.claimed + o) < p.vcount[o] &&
                (j == 0 || pk_ld(p.done + o - 1) >= p.vcount[o - 1] + probe);
      }
    }
    if (__any_sync(0xffffffffu, c < p.nctx && j < p.ctx_nops[c])) all_finished = false;
    unsigned ballot = __ballot_sync(0xffffffffu, ready);
    while (ballot) {
      const int src = __ffs(ballot) - 1;
      const int oc = __shfl_sync(0xffffffffu, o, src);
      const int jc = __shfl_sync(0xffffffffu, j, src);
      int got = -1;
      if (lane == 0) {
        const int it = atomicAdd(p.claimed + oc, 1);
        const int cnt = p.vcount[oc];
        if (it >= cnt - 1) atomicMax(p.cur + base + src, jc + 1);  // the op is fully handed out
        if (it < cnt) {
          got = oc;
          *item = it;
        }
      }
      got = __shfl_sync(0xffffffffu, got, 0);
      if (got >= 0) return got;
      ballot &= ballot - 1;
    }
  }
  return all_finished ? -2 : -1;
}

template <bool F32, bool AC, bool BC, int G>
__device__ __forceinline__ void pk_spmm_g(const PkSpmm& o, const Cta& c) {
  using T = typename std::conditional<F32, float, double>::type;
  using VR = typename std::conditional<F32, float, double>::type;
  using VCx = typename std::conditional<F32, float2, double2>::type;
  using VA = typename std::conditional<AC, VCx, VR>::type;
  using VB = typename std::conditional<BC, VCx, VR>::type;
  constexpr int V = F32 ? 2 : 1;
  CsrDev<VA> a{o.arp, o.acol, (const VA*)o.aval};
  CsrDev<VB> b{o.brp, o.bcol, (const VB*)o.bval};
  spmm_body<VA, VB, T, G, V, false>(c, o.n, a, b, o.hasB, (const cplx<T>*)o.X, o.ldx, o.w, o.AX, o.ldax, o.BX,
                                    o.ldbx);
}

template <bool F32, bool AC, bool BC>
__device__ __forceinline__ void pk_spmm_gi(int gi, const PkSpmm& o, const Cta& c) {
  switch (gi) {
    case 0: pk_spmm_g<F32, AC, BC, 4>(o, c); break;
    case 1: pk_spmm_g<F32, AC, BC, 8>(o, c); break;
    case 2: pk_spmm_g<F32, AC, BC, 16>(o, c); break;
    default: pk_spmm_g<F32, AC, BC, 32>(o, c); break;
  }
}

__device__ __forceinline__ void pk_spmm(int code, const PkSpmm& o, const Cta& c) {
  const int gi = code >> 3;
  switch (code & 7) {
    case 0: pk_spmm_gi<false, false, false>(gi, o, c); break;
    case 1: pk_spmm_gi<true, false, false>(gi, o, c); break;
    case 2: pk_spmm_gi<false, true, false>(gi, o, c); break;
    case 3: pk_spmm_gi<true, true, false>(gi, o, c); break;
    case 4: pk_spmm_gi<false, false, true>(gi, o, c); break;
    case 5: pk_spmm_gi<true, false, true>(gi, o, c); break;
    case 6: pk_spmm_gi<false, true, true>(gi, o, c); break;
    default: pk_spmm_gi<true, true, true>(gi, o, c); break;
  }
}

template <int ACC>
__device__ __forceinline__ void pk_gram_acc(int mode, const PkGram& o, const Cta& c) {
  if (mode == 2)
    gram_partial_x32_body<ACC>(c, o.n, o.rows, o.X, o.ldx, o.wx, o.Y0, o.ldy0, o.wy0, o.Y1, o.ldy1, o.wy1, o.herm,
                               o.nout, o.G, o.RG, o.partial, o.skip);
  else if (mode == 1)
    gram_partial_body<ACC, float>(c, o.n, o.rows, o.X, o.ldx, o.wx, o.Y0, o.ldy0, o.wy0, o.Y1, o.ldy1, o.wy1,
                                  o.herm, o.nout, o.G, o.RG, o.partial, o.skip);
  else
    gram_partial_body<ACC, double>(c, o.n, o.rows, o.X, o.ldx, o.wx, o.Y0, o.ldy0, o.wy0, o.Y1, o.ldy1, o.wy1,
                                   o.herm, o.nout, o.G, o.RG, o.partial, o.skip);
}

__device__ __forceinline__ void pk_run(int kind, const unsigned char* arg, const Cta& c) {
  if (kind >= PK_SPMM_BASE) {
    pk_spmm(kind - PK_SPMM_BASE, *reinterpret_cast<const PkSpmm*>(arg), c);
    return;
  }
  if (kind >= PK_GRAM_BASE) {
    const PkGram& o = *reinterpret_cast<const PkGram*>(arg);
    const int mode = (kind - PK_GRAM_BASE) >> 2, lacc = (kind - PK_GRAM_BASE) & 3;
    switch (lacc) {
      case 0: pk_gram_acc<1>(mode, o, c); break;
      case 1: pk_gram_acc<2>(mode, o, c); break;
      case 2: pk_gram_acc<4>(mode, o, c); break;
      default: pk_gram_acc<8>(mode, o, c); break;
    }
    return;
  }
  switch (kind) {
    case PK_BYTES: {
      const PkBytes& o = *reinterpret_cast<const PkBytes*>(arg);
      for (int64_t e = (int64_t)c.x * PK_THREADS + threadIdx.x; e < o.count; e += (int64_t)c.gx * PK_THREADS)
        o.dst[e] = o.src[e];
      break;
    }
    case PK_COPY_RAW: {  // 16-byte words where both ends allow, else bytes
      const PkRaw& o = *reinterpret_cast<const PkRaw*>(arg);
      const int64_t t0 = (int64_t)c.x * PK_THREADS + threadIdx.x, nt = (int64_t)c.gx * PK_THREADS;
      if ((((uintptr_t)o.src | (uintptr_t)o.dst | (uintptr_t)o.bytes) & 15) == 0) {
        const int4* s4 = reinterpret_cast<const int4*>(o.src);
        int4* d4 = reinterpret_cast<int4*>(o.dst);
        for (int64_t e = t0; e < o.bytes / 16; e += nt) d4[e] = s4[e];
      } else {
        for (int64_t e = t0; e < o.bytes; e += nt) o.dst[e] = o.src[e];
      }
      break;
    }
    case PK_AXPBY: {
      const PkAxpby& o = *reinterpret_cast<const PkAxpby*>(arg);
      axpby_body(c, o.n, o.w, o.alpha, o.X1, o.ld1, o.beta, o.X2, o.ld2, o.Y, o.ldy);
      break;
    }
    case PK_COPY_BLOCK: {
      const PkCopy& o = *reinterpret_cast<const PkCopy*>(arg);
      copy_block_body(c, o.n, o.w, o.X, o.ldx, o.Y, o.ldy);
      break;
    }
    case PK_TO_C64: {
      const PkToC64& o = *reinterpret_cast<const PkToC64*>(arg);
      to_c64_body(c, o.n, o.w, o.X, o.ldx, o.Y, o.ldy);
      break;
    }
    case PK_GRAM_REDUCE: {
      const PkGramRed& o = *reinterpret_cast<const PkGramRed*>(arg);
      gram_reduce_body(c, o.nchunk, o.nout, o.wx, o.wy, o.herm, o.partial, o.C, o.ldc, o.skip);
      break;
    }
    case PK_NORM_REDUCE: {
      const PkNormRed& o = *reinterpret_cast<const PkNormRed*>(arg);
      norm_reduce_body(c, o.nb, o.nc, o.part, o.out);
      break;
    }
    case PK_CHOL: {
      const PkChol& o = *reinterpret_cast<const PkChol*>(arg);
      chol_inv_body(c, o.w, o.n, o.G, o.Rinv, o.status, o.skip, o.fallback, o.Rout, o.work);
      break;
    }
    case PK_COMBINE_D: {
      const PkComb& o = *reinterpret_cast<const PkComb*>(arg);
      combine_body<double>(c, o.n, o.rows_per_cta, o.a);
      break;
    }
    case PK_COMBINE_F: {
      const PkComb& o = *reinterpret_cast<const PkComb*>(arg);
      combine_body<float>(c, o.n, o.rows_per_cta, o.a);
      break;
    }
    case PK_JACOBI_D:
    case PK_JACOBI_F: {
      const PkJacobi& o = *reinterpret_cast<const PkJacobi*>(arg);
      if (kind == PK_JACOBI_D)
        jacobi_body<double>(c, o.n, o.w, o.d, o.X, o.ldx, o.Y, o.ldy);
      else
        jacobi_body<float>(c, o.n, o.w, o.d, o.X, o.ldx, o.Y, o.ldy);
      break;
    }
    case PK_BJ_DD: {
      const PkBj& o = *reinterpret_cast<const PkBj*>(arg);
      block_jacobi_body<double, double2>(c, o.n, o.bs, o.w, (const double2*)o.Tinv, o.X, o.ldx, o.Y, o.ldy, o.bpc);
      break;
    }
    case PK_BJ_FD: {
      const PkBj& o = *reinterpret_cast<const PkBj*>(arg);
      block_jacobi_body<float, double2>(c, o.n, o.bs, o.w, (const double2*)o.Tinv, o.X, o.ldx, o.Y, o.ldy, o.bpc);
      break;
    }
    case PK_BJ_FF: {
      const PkBj& o = *reinterpret_cast<const PkBj*>(arg);
      block_jacobi_body<float, float2>(c, o.n, o.bs, o.w, (const float2*)o.Tinv, o.X, o.ldx, o.Y, o.ldy, o.bpc);
      break;
    }
    default:
      break;
  }
}

// The persistent kernel: claim a ready item, run it, count it finished; sleep when nothing
// is ready; return when every context has finished or a wait ran out.
__global__ void __launch_bounds__(PK_THREADS, PK_CTAS_PER_SM)
persistent_segment_kernel(PkProgram p, PkQueue* q, int* err, unsigned long long limit_ns, int probe) {
  __shared__ int s_op, s_item;
  unsigned long long idle_since = 0;
  for (;;) {
    if (threadIdx.x < 32) {
      int item = 0;
      int op = *(volatile int*)&q->abort ? -2 : pk_claim(p, probe, &item);
      if (threadIdx.x == 0) {
        if (op >= 0) {
          __threadfence();  // the previous op's writes (its items fence before counting) before ours
          idle_since = 0;
        } else if (op == -1) {
          const unsigned long long t = pk_globaltimer();
          if (idle_since == 0) idle_since = t;
          if (t - idle_since > limit_ns) {
            atomicExch(&q->abort, 1);
            atomicCAS(err, 0, 7);
            op = -2;
          }
        }
        s_op = op;
        s_item = item;
      }
    }
    __syncthreads();
    const int o = s_op, it = s_item;
    if (o == -2) return;
    if (o == -1) {
      if (threadIdx.x == 0) __nanosleep(256);
      __syncthreads();
      continue;
    }
    const PkOp op = p.ops[o];
    const Cta c{it % op.gx, it / op.gx, op.gx, op.gy};
    pk_run(op.kind, p.args + op.argoff, c);
    __syncthreads();  // the item's writes are done (and the next item reuses shared memory)
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(p.done + o, 1);
    }
  }
}

}  // namespace gplhr
