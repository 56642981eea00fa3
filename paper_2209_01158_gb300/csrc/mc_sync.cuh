// Grid-wide synchronisation and deterministic reductions for the persistent
// (cooperative) kernels of libmc.so.
//
// The barrier is a monotonic 64-bit arrival counter: barrier number b is
// passed when the counter reaches (b + 1) * G, G the CTAs taking part (the
// whole grid, or one team of the batched kernel), so one release atomic
// per CTA and acquire polls suffice (no reset, no generation word). Every
// wait is bounded by `spin_limit` polls; a CTA that gives up raises the abort
// word and the status MC_E_TIMEOUT, and CTAs that see the abort word while
// waiting leave too, so no launch can hang.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mc.h"

struct GridBar {
  unsigned long long* count = nullptr;  // zeroed before the launch
  unsigned* abort_word = nullptr;       // zeroed before the launch
  int* status = nullptr;
  long long spin_limit = 0;
  unsigned nparts = 0;                  // CTAs taking part (0: the whole grid)
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long atom_add_release_u64(unsigned long long* p,
                                                                   unsigned long long v) {
  unsigned long long old;
  asm volatile("atom.add.release.gpu.global.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
  return old;
}

__device__ __forceinline__ void grid_raise_abort(const GridBar& g, int code) {
  atomicExch(g.abort_word, 1u);
  atomicCAS(g.status, 0, code);
}

// Returns false when the launch must stop (timeout here or abort elsewhere).
// Thread 0 of each CTA does the arrival; the rest wait at the CTA barrier.
__device__ __forceinline__ bool grid_barrier(const GridBar& g) {
  __shared__ int s_grid_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    const unsigned long long G = g.nparts ? g.nparts : gridDim.x;
    const unsigned long long old = atom_add_release_u64(g.count, 1ull);
    const unsigned long long target = (old / G + 1ull) * G;
    long long n = 0;
    while (ld_acquire_u64(g.count) < target) {
      ++n;
      if ((n & 63) == 0 && ld_acquire_u32(g.abort_word) != 0u) { ok = 0; break; }
      if (n > g.spin_limit) {
        grid_raise_abort(g, (int)MC_E_TIMEOUT);
        ok = 0;
        break;
      }
      __nanosleep(20);
    }
    s_grid_ok = ok;
  }
  __syncthreads();
  return s_grid_ok != 0;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic CTA sum of NQ values; every thread receives the totals.
// s_red needs (blockDim.x / 32) * NQ doubles, s_res NQ doubles.
template <int NQ>
__device__ __forceinline__ void cta_sum(double (&v)[NQ], double* s_red, double* s_res) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NQ; ++k) {
    const double s = warp_sum_d(v[k]);
    if (lane == 0) s_red[warp * NQ + k] = s;
  }
  __syncthreads();
  if (threadIdx.x < NQ) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += s_red[w * NQ + threadIdx.x];
    s_res[threadIdx.x] = s;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NQ; ++k) v[k] = s_res[k];
  __syncthreads();
}

// Deterministic CTA reduction of NQ per-thread partial sums, stored as this
// CTA's entries partials[(slot * KM + k) * gridDim.x + blockIdx.x].
// The values are staged through shared memory (8 quantities at a time) and
// each quantity is summed by ONE warp: 16 adds per lane and a 5-level
// butterfly, instead of a butterfly in every warp. On GB300 a 32-lane FP64
// instruction costs about 16 issue cycles per SM, so this cuts the FP64 work
// of a reduction about fourfold. Quantities whose bit is clear in qmask are
// skipped and stored as 0. `stage` needs 8 * NTH elements.
template <int NQ, int NTH, int KM, typename T>
__device__ __forceinline__ void cta_reduce_store(const T (&v)[NQ], unsigned qmask, T* stage,
                                                 double* partials, int slot, int nb = -1,
                                                 int b = -1) {
  if (nb < 0) {
    nb = gridDim.x;
    b = blockIdx.x;
  }
  static_assert(NTH % 32 == 0 && NTH >= 256, "block size");
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int c0 = 0; c0 < NQ; c0 += 8) {
#pragma unroll
    for (int k = c0; k < NQ && k < c0 + 8; ++k)
      if (qmask & (1u << k)) stage[(k - c0) * NTH + tid] = v[k];
    __syncthreads();
    const int k = c0 + warp;
    if (warp < 8 && k < NQ) {
      T s = T(0);
      if (qmask & (1u << k)) {
        const T* col = stage + (k - c0) * NTH;
#pragma unroll
        for (int j = 0; j < NTH / 32; ++j) s += col[lane + 32 * j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      }
      if (lane == 0) partials[((size_t)slot * KM + k) * nb + b] = (double)s;
    }
    __syncthreads();
  }
}

// qmask with bit q*L + a set for every a in `mask` and q < nq.
__device__ __forceinline__ unsigned qbits(unsigned mask, int L, int nq) {
  unsigned m = 0;
  for (int q = 0; q < nq; ++q) m |= mask << (q * L);
  return m;
}
