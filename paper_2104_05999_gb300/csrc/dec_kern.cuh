// dec_kern.cuh - device building blocks shared by the solver kernels:
// mixed-type FMA helpers and the SELL-32-512 row product.  Internal.
#pragma once

#include "dec_internal.cuh"

namespace dec {

__device__ __forceinline__ double to_d(double v) { return v; }
__device__ __forceinline__ double to_d(float v) { return (double)v; }

__device__ __forceinline__ double fma_(double a, double x, double acc) { return fma(a, x, acc); }
__device__ __forceinline__ float fma_(float a, float x, float acc) { return fmaf(a, x, acc); }
__device__ __forceinline__ float fma_(__nv_bfloat16 a, float x, float acc) {
  return fmaf(__bfloat162float(a), x, acc);
}

// Matrix in SELL form, as kernel arguments.
template <typename T>
struct SellArg {
  const int32_t* perm;
  const int32_t* sptr;
  const int32_t* col;
  const T* val;
  int64_t nslices;
};

template <typename T>
inline SellArg<T> sell_arg(const SellLayout& L, const T* val) {
  return SellArg<T>{L.perm.p, L.sptr.p, L.col.p, val, L.nslices};
}

// Row sum of the lane's row in slice s: sum_j val * x[col].  Entries are
// taken 8 at a time: 8 column and 8 value loads, then 8 independent gathers,
// then the FMAs, so each warp keeps many loads in flight (the width w is
// uniform across the warp, so the guards never diverge).
template <typename MT, typename VT, int U = 8>
__device__ __forceinline__ VT sell_row(const SellArg<MT>& A, int64_t s, int lane,
                                       const VT* __restrict__ x) {
  const int32_t base = __ldg(A.sptr + s);
  const int32_t w = (__ldg(A.sptr + s + 1) - base) >> 5;
  const int32_t* __restrict__ cp = A.col + base + lane;
  const MT* __restrict__ vp = A.val + base + lane;
  VT acc = VT(0);
  for (int32_t j = 0; j < w; j += U) {
    int32_t c[U];
    MT a[U];
    VT xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const bool ok = j + u < w;
      c[u] = ok ? __ldg(cp + 32 * (j + u)) : 0;
      a[u] = ok ? vp[32 * (j + u)] : MT(0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) xv[u] = j + u < w ? __ldg(x + c[u]) : VT(0);
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (j + u < w) acc = fma_(a[u], xv[u], acc);   // uniform: no idle FMAs
  }
  return acc;
}

// 16-byte asynchronous global -> shared copy (L2 only) and its wait.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// Shared-memory bytes one warp needs to stage WMAX entries of a slice
// (32 columns and 32 values per entry).
template <int WMAX, typename MT>
__host__ __device__ constexpr int stage_bytes() {
  return WMAX * 32 * (int)(sizeof(int32_t) + sizeof(MT));
}

// sell_row with the slice's columns and values first copied to the warp's
// shared-memory stage in one burst of 16-byte asynchronous copies, so the
// whole slice is in flight at once and the row loop only waits on the
// gathers of x.  Entries beyond WMAX (rare wide slices) are read from global
// memory.  `stage` is this warp's region of stage_bytes<WMAX, MT>() bytes,
// 16-byte aligned.
template <int WMAX, typename MT, typename VT>
__device__ __forceinline__ VT sell_row_staged(const SellArg<MT>& A, int64_t s, int lane,
                                              const VT* __restrict__ x,
                                              unsigned char* stage) {
  constexpr int U = 8;
  const int32_t base = __ldg(A.sptr + s);
  const int32_t w = (__ldg(A.sptr + s + 1) - base) >> 5;
  const int32_t ws = w < WMAX ? w : WMAX;
  int32_t* scol = reinterpret_cast<int32_t*>(stage);
  MT* sval = reinterpret_cast<MT*>(stage + WMAX * 32 * sizeof(int32_t));
  {
    // columns: 128 B per entry; values: 32 * sizeof(MT) B per entry
    const unsigned char* gc = reinterpret_cast<const unsigned char*>(A.col + base);
    const int nc = ws * 8;
    for (int k = lane; k < nc; k += 32) cp_async16(stage + 16 * k, gc + 16 * k);
    const unsigned char* gv = reinterpret_cast<const unsigned char*>(A.val + base);
    unsigned char* sv = reinterpret_cast<unsigned char*>(sval);
    const int nv = ws * 2 * (int)sizeof(MT);
    for (int k = lane; k < nv; k += 32) cp_async16(sv + 16 * k, gv + 16 * k);
    cp_async_wait_all();
    __syncwarp();
  }
  VT acc = VT(0);
  for (int32_t j = 0; j < w; j += U) {
    int32_t c[U];
    VT xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int32_t e = j + u;
      c[u] = e < ws ? scol[32 * e + lane] : (e < w ? __ldg(A.col + base + 32 * e + lane) : 0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) xv[u] = j + u < w ? __ldg(x + c[u]) : VT(0);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int32_t e = j + u;
      if (e < w) {
        const MT a = e < ws ? sval[32 * e + lane] : A.val[base + 32 * e + lane];
        acc = fma_(a, xv[u], acc);
      }
    }
  }
  __syncwarp();   // the stage is reused by the warp's next slice
  return acc;
}

}  // namespace dec
