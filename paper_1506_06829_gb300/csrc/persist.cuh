// Persistent kernel of the batched iteration: one launch runs a whole device segment of
// an iteration (Algorithm 2, steps 7-24, steps 25-28, or the residual with its column
// norms) for every context of a batch.
//
// The host records each context's segment as the list of launches it would make (kernel,
// grid, arguments), in program order.  Step j of the program is the j-th recorded launch
// of every context that has one; the kernel walks the steps, spreads the CTAs of each
// step's launches (their "virtual" CTAs) over its own CTAs, runs each virtual CTA with
// the body of the recorded kernel, and crosses a grid-wide barrier before the next step.
// A launch depends only on the earlier launches of its own context, so one barrier per
// step keeps every context's order while the contexts' launches run side by side.
//
// Launched cooperatively (all CTAs resident), so the barrier always completes; its wait
// is bounded all the same (a time limit on the global timer), after which the kernel
// records GPLHR_ETIMEOUT and every CTA returns at its next barrier.
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

// Device program: ops sorted by step; step j holds ops [step_begin[j], step_begin[j+1]);
// vstart[o] = first virtual CTA of op o within its step, step_total[j] = the step's count.
struct PkProgram {
  const PkOp* ops;
  const unsigned char* args;
  const int* step_begin;
  const int* vstart;
  const int* step_total;
  int nsteps;
};

// Barrier state, zeroed by the host before each launch.
struct PkBarrier {
  unsigned count;
  unsigned gen;
  int abort;
  int pad;
};

__device__ __forceinline__ unsigned long long pk_globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier (sense by generation count).  Thread 0 of each CTA publishes the
// CTA's writes (fence), arrives, and waits for the generation to move on; the last
// arrival opens it.  The wait is bounded by limit_ns of global time: then the abort flag
// is raised, err records GPLHR_ETIMEOUT (7) and every CTA leaves at this or its next
// barrier.  probe (test hook): the last arrival does not open the barrier, so the wait
// runs out.  Returns false when the kernel must end.
__device__ __forceinline__ bool pk_grid_barrier(PkBarrier* b, unsigned nblocks, int* err,
                                                unsigned long long limit_ns, int probe) {
  __shared__ int pk_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = &b->gen;
    volatile int* vabort = &b->abort;
    const unsigned g = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(&b->count, 1u);
    if (arrived == nblocks - 1 && !probe) {
      atomicExch(&b->count, 0u);
      __threadfence();
      atomicAdd(&b->gen, 1u);
    } else {
      const unsigned long long t0 = pk_globaltimer();
      while (*vgen == g && !*vabort) {
        if (pk_globaltimer() - t0 > limit_ns) {
          atomicExch(&b->abort, 1);
          atomicCAS(err, 0, 7);
          break;
        }
        __nanosleep(128);
      }
    }
    __threadfence();
    pk_ok = *vabort ? 0 : 1;
  }
  __syncthreads();
  return pk_ok != 0;
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

// The persistent kernel: one program, every step's virtual CTAs over this grid, a bounded
// grid barrier between steps.
__global__ void __launch_bounds__(PK_THREADS, PK_CTAS_PER_SM)
persistent_segment_kernel(PkProgram p, PkBarrier* bar, int* err, unsigned long long limit_ns, int probe) {
  for (int j = 0; j < p.nsteps; ++j) {
    const int o0 = p.step_begin[j], o1 = p.step_begin[j + 1];
    const int total = p.step_total[j];
    for (int v = blockIdx.x; v < total; v += gridDim.x) {
      int lo = o0, hi = o1 - 1;  // last op of the step whose first virtual CTA is <= v
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (p.vstart[mid] <= v) lo = mid; else hi = mid - 1;
      }
      const PkOp op = p.ops[lo];
      const int local = v - p.vstart[lo];
      const Cta c{local % op.gx, local / op.gx, op.gx, op.gy};
      pk_run(op.kind, p.args + op.argoff, c);
      __syncthreads();  // the next virtual CTA reuses shared memory
    }
    if (j + 1 < p.nsteps && !pk_grid_barrier(bar, gridDim.x, err, limit_ns, probe)) return;
  }
}

}  // namespace gplhr
