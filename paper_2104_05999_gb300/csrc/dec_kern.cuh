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
template <typename MT, typename VT>
__device__ __forceinline__ VT sell_row(const SellArg<MT>& A, int64_t s, int lane,
                                       const VT* __restrict__ x) {
  constexpr int U = 8;
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

}  // namespace dec

