// dec_sort.cu - exclusive prefix sum and stable LSD radix sort of
// (uint64 key, uint32 value) pairs.  These order the 6 edge keys of every
// tet (to extract the unique edges, i.e. the sparsity of d0) and the
// transposed edge list (to build the CSR rows of L without atomics).
#include "dec_internal.cuh"

namespace dec {

// ------------------------------------------------------------ prefix sum
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__global__ void __launch_bounds__(kScanThreads)
scan_reduce_kernel(const uint32_t* __restrict__ in, uint32_t* __restrict__ bsum,
                   int64_t n) {
  __shared__ uint32_t sh[32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
    if (i < n) s += in[i];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    uint32_t t = threadIdx.x < kScanThreads / 32 ? sh[threadIdx.x] : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) bsum[blockIdx.x] = t;
  }
}

// Exclusive scan of the block sums by one block, chunk by chunk.
__global__ void __launch_bounds__(1024) scan_top_kernel(uint32_t* a, int64_t n) {
  __shared__ uint32_t warp_tot[32];
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int64_t base = 0; base < n; base += 1024) {
    int64_t i = base + threadIdx.x;
    uint32_t v = i < n ? a[i] : 0u;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      uint32_t t = warp_tot[lane];
      uint32_t ti = t;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t u = __shfl_up_sync(0xffffffffu, ti, o);
        if (lane >= o) ti += u;
      }
      warp_tot[lane] = ti - t;  // exclusive over warps
    }
    __syncthreads();
    uint32_t excl = carry + warp_tot[wid] + incl - v;
    if (i < n) a[i] = excl;
    __syncthreads();
    if (threadIdx.x == 1023) carry = excl + v;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kScanThreads)
scan_down_kernel(const uint32_t* in, uint32_t* out,
                 const uint32_t* __restrict__ boff, int64_t n) {
  __shared__ uint32_t warp_tot[kScanThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile +
                       (int64_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = base + k;
    v[k] = i < n ? in[i] : 0u;
    s += v[k];
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  uint32_t wofs = 0;
  for (int w = 0; w < wid; ++w) wofs += warp_tot[w];
  uint32_t run = boff[blockIdx.x] + wofs + incl - s;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = base + k;
    if (i < n) out[i] = run;
    run += v[k];
  }
}

size_t scan_tmp_size(int64_t n) { return (size_t)((n + kScanTile - 1) / kScanTile) + 1; }

// out[i] = sum_{k < i} in[k]; in == out is allowed.  `tmp` needs
// scan_tmp_size(n) entries.
cudaError_t exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n,
                               uint32_t* tmp, size_t tmp_cap, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int64_t nb = (n + kScanTile - 1) / kScanTile;
  if ((size_t)nb > tmp_cap) return cudaErrorInvalidValue;
  scan_reduce_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(in, tmp, n);
  scan_top_kernel<<<1, 1024, 0, s>>>(tmp, nb);
  scan_down_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, tmp, n);
  return cudaGetLastError();
}

// ------------------------------------------------------------ radix sort
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortRounds = 16;                  // 32 items per warp round
constexpr int kSortTile = kSortThreads * kSortRounds;   // 4096 pairs
constexpr int kRadix = 256;

__global__ void __launch_bounds__(kSortThreads)
radix_hist_kernel(const uint64_t* __restrict__ keys, int64_t n, int shift,
                  uint32_t* __restrict__ hist, int tiles) {
  __shared__ uint32_t cnt[kRadix];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
#pragma unroll 4
  for (int k = 0; k < kSortRounds; ++k) {
    int64_t i = base + (int64_t)k * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&cnt[(unsigned)(keys[i] >> shift) & (kRadix - 1)], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * tiles + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter: warp w owns tile items [w*512, w*512+512) and walks them
// in order, 32 at a time; items of equal digit keep their order through
// per-warp digit counters and an exclusive prefix over warps.
__global__ void __launch_bounds__(kSortThreads)
radix_scatter_kernel(const uint64_t* __restrict__ keys,
                     const uint32_t* __restrict__ vals, int64_t n, int shift,
                     const uint32_t* __restrict__ offs, int tiles,
                     uint64_t* __restrict__ keys_out,
                     uint32_t* __restrict__ vals_out) {
  __shared__ uint32_t wcnt[kSortWarps][kRadix];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int d = threadIdx.x; d < kSortWarps * kRadix; d += kSortThreads)
    (&wcnt[0][0])[d] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kSortTile +
                       (int64_t)wid * (kSortRounds * 32);
  uint64_t k_reg[kSortRounds];
  uint32_t v_reg[kSortRounds];
  uint32_t rank[kSortRounds];
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r) {
    int64_t i = base + r * 32 + lane;
    bool ok = i < n;
    k_reg[r] = ok ? keys[i] : 0ull;
    v_reg[r] = ok ? vals[i] : 0u;
    unsigned valid = __ballot_sync(0xffffffffu, ok);
    unsigned d = ok ? (unsigned)(k_reg[r] >> shift) & (kRadix - 1) : kRadix;
    unsigned peers = __match_any_sync(0xffffffffu, d) & valid;
    uint32_t before = ok ? wcnt[wid][d] : 0u;
    rank[r] = before + __popc(peers & lt);
    __syncwarp();
    if (ok && (peers & lt) == 0) wcnt[wid][d] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  {  // exclusive prefix of the per-warp counts, per digit
    const int d = threadIdx.x;
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) {
      uint32_t t = wcnt[w][d];
      wcnt[w][d] = run;
      run += t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r) {
    int64_t i = base + r * 32 + lane;
    if (i < n) {
      unsigned d = (unsigned)(k_reg[r] >> shift) & (kRadix - 1);
      uint32_t pos = offs[(int64_t)d * tiles + blockIdx.x] + wcnt[wid][d] + rank[r];
      keys_out[pos] = k_reg[r];
      vals_out[pos] = v_reg[r];
    }
  }
}

// Sort n pairs by the low `key_bits` bits of the key (stable).  The result is
// in (keys, vals) or, when *result_in_alt, in (keys_alt, vals_alt).
dec_status radix_sort_pairs(dec_ctx* ctx, uint64_t* keys, uint32_t* vals,
                            uint64_t* keys_alt, uint32_t* vals_alt, int64_t n,
                            int key_bits, bool* result_in_alt) {
  *result_in_alt = false;
  if (n <= 1) return DEC_OK;
  if (n >= (int64_t)1 << 32) return ctx->fail(DEC_ERR_LIMIT, "sort: too many pairs");
  const int tiles = (int)((n + kSortTile - 1) / kSortTile);
  const int64_t hn = (int64_t)tiles * kRadix;
  DEC_TRY(ctx->hist.ensure(hn));
  DEC_TRY(ctx->scan_tmp.ensure(scan_tmp_size(hn)));
  const int passes = (key_bits + 7) / 8;
  uint64_t *ki = keys, *ko = keys_alt;
  uint32_t *vi = vals, *vo = vals_alt;
  for (int p = 0; p < passes; ++p) {
    const int shift = 8 * p;
    radix_hist_kernel<<<tiles, kSortThreads, 0, ctx->stream>>>(ki, n, shift, ctx->hist.p, tiles);
    ctx->launches += 5;  // histogram, 3-kernel scan, scatter
    DEC_TRY(exclusive_scan_u32(ctx->hist.p, ctx->hist.p, hn, ctx->scan_tmp.p,
                               ctx->scan_tmp.cap, ctx->stream));
    radix_scatter_kernel<<<tiles, kSortThreads, 0, ctx->stream>>>(
        ki, vi, n, shift, ctx->hist.p, tiles, ko, vo);
    DEC_TRY(cudaGetLastError());
    std::swap(ki, ko);
    std::swap(vi, vo);
    *result_in_alt = !*result_in_alt;
  }
  return DEC_OK;
}

}  // namespace dec
