// Persistent kernel of the batched iteration: one launch runs a whole device segment of
// an iteration (Algorithm 2, steps 7-24, steps 25-28, or the residual with its column
// norms) for every context of a batch.
//
// The host records each context's segment as the list of launches it would make (kernel,
// grid, arguments), in program order, and merges the lists into one queue: the j-th
// launches of all contexts, then the (j+1)-th, and so on, each launch as its grid's
// "virtual" CTAs.  The kernel's CTAs take queue items in order from a global counter; an
// item first waits until the previous launch of its own context has finished (a count of
// its finished virtual CTAs), then runs the recorded kernel's body for its virtual CTA and
// counts itself finished.  A launch depends only on the earlier launches of its context,
// so the contexts advance independently: a slow step of one (a Cholesky factorisation, a
// large Gram product) does not hold up the others.  Every item waits only on items earlier
// in the queue, which are held by running CTAs, so the waits always end.
//
// Launched cooperatively (all CTAs resident); every wait is bounded all the same (a time
// limit on the global timer), after which the kernel records GPLHR_ETIMEOUT and every CTA
// returns.
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
};
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

// Device program: ops in queue order (the j-th launches of all contexts before the
// (j+1)-th); op o owns queue items vstart[o] .. vstart[o+1] - 1 (its virtual CTAs), waits
// for op prev[o] (its context's previous launch, -1 for none), and counts its finished
// items in done[o] (zeroed before each launch).
struct PkProgram {
  const PkOp* ops;
  const unsigned char* args;
  const int* vstart;  // nops + 1 entries
  const int* prev;
  int* done;
  int nops;
};

// Queue state, zeroed by the host before each launch.
struct PkQueue {
  unsigned next;
  int abort;
  int pad[2];
};

__device__ __forceinline__ unsigned long long pk_globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Thread 0 of the CTA: wait until op d has finished `need` virtual CTAs.  Bounded by
// limit_ns of global time: then the abort flag is raised, err records GPLHR_ETIMEOUT (7),
// and false is returned (also when another CTA has aborted).  The fence after the wait
// orders the CTA's later reads after the producers' writes (they fence before counting).
__device__ __forceinline__ bool pk_wait_done(const int* done, int need, PkQueue* q, int* err,
                                             unsigned long long limit_ns) {
  volatile const int* vd = done;
  volatile int* vabort = &q->abort;
  if (*vd < need) {
    const unsigned long long t0 = pk_globaltimer();
    while (*vd < need) {
      if (*vabort) return false;
      if (pk_globaltimer() - t0 > limit_ns) {
        atomicExch(&q->abort, 1);
        atomicCAS(err, 0, 7);
        return false;
      }
      __nanosleep(64);
    }
  }
  __threadfence();
  return true;
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
      chol_inv_body(c, o.w, o.n, o.G, o.Rinv, o.status, o.skip, o.fallback, o.Rout);
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

// The persistent kernel: CTAs take queue items in order, wait for their context's previous
// launch, run the item's virtual CTA and count it finished.  probe (test hook): every wait
// asks for one virtual CTA more than its op has, so the first wait runs out.
__global__ void __launch_bounds__(PK_THREADS, PK_CTAS_PER_SM)
persistent_segment_kernel(PkProgram p, PkQueue* q, int* err, unsigned long long limit_ns, int probe) {
  __shared__ int s_item, s_ok;
  const int total = p.vstart[p.nops];
  for (;;) {
    if (threadIdx.x == 0) {
      const volatile int* vabort = &q->abort;
      s_item = *vabort ? total : (int)atomicAdd(&q->next, 1u);
    }
    __syncthreads();
    const int v = s_item;
    if (v >= total) return;
    int lo = 0, hi = p.nops - 1;  // the op owning item v: last op with vstart <= v
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (p.vstart[mid] <= v) lo = mid; else hi = mid - 1;
    }
    if (threadIdx.x == 0) {
      const int d = p.prev[lo];
      s_ok = d < 0 ? 1 : (pk_wait_done(p.done + d, p.vstart[d + 1] - p.vstart[d] + (probe ? 1 : 0), q, err,
                                       limit_ns) ? 1 : 0);
    }
    __syncthreads();
    if (!s_ok) return;
    const PkOp op = p.ops[lo];
    const int local = v - p.vstart[lo];
    const Cta c{local % op.gx, local / op.gx, op.gx, op.gy};
    pk_run(op.kind, p.args + op.argoff, c);
    __syncthreads();  // the item's writes are done (and the next item reuses shared memory)
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(p.done + lo, 1);
    }
  }
}

}  // namespace gplhr
