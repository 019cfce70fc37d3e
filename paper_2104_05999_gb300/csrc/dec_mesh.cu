// dec_mesh.cu - mesh validation, the edge list of the tetrahedral complex
// (the rows of the incidence matrix d0, Sec. 2.1) and the CSR structure of
// L = d0^T *1 d0, all integer work, built without atomics from sorted keys.
#include "dec_internal.cuh"

namespace dec {

__constant__ int kLocalEdge[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};

// ----------------------------------------------------------- validation
// errflag bit 1: node id out of range, bit 2: tet not positively oriented,
// bit 4: bad node tag.
__global__ void validate_tets_kernel(const int32_t* __restrict__ tets,
                                     const double* __restrict__ xyz, int64_t m,
                                     int64_t n, int* errflag) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m;
       t += (int64_t)gridDim.x * blockDim.x) {
    int4 v = reinterpret_cast<const int4*>(tets)[t];
    if (v.x < 0 || v.y < 0 || v.z < 0 || v.w < 0 || v.x >= n || v.y >= n ||
        v.z >= n || v.w >= n) {
      atomicOr(errflag, 1);
      continue;
    }
    const double* p0 = xyz + 3 * (int64_t)v.x;
    const double* p1 = xyz + 3 * (int64_t)v.y;
    const double* p2 = xyz + 3 * (int64_t)v.z;
    const double* p3 = xyz + 3 * (int64_t)v.w;
    double ax = p1[0] - p0[0], ay = p1[1] - p0[1], az = p1[2] - p0[2];
    double bx = p2[0] - p0[0], by = p2[1] - p0[1], bz = p2[2] - p0[2];
    double cx = p3[0] - p0[0], cy = p3[1] - p0[1], cz = p3[2] - p0[2];
    double det = ax * (by * cz - bz * cy) + ay * (bz * cx - bx * cz) +
                 az * (bx * cy - by * cx);
    if (!(det > 0.0)) atomicOr(errflag, 2);
  }
}

__global__ void validate_tags_kernel(const uint8_t* __restrict__ tag, int64_t n,
                                     int* errflag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (tag[i] > 2) atomicOr(errflag, 4);
}

// ------------------------------------------------------------ edge list
// key of the directed-once edge (i, j), i < j: i * n + j; value: tet*6+slot.
__global__ void edge_keys_kernel(const int32_t* __restrict__ tets, int64_t m,
                                 int64_t n, uint64_t* __restrict__ keys,
                                 uint32_t* __restrict__ vals) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m;
       t += (int64_t)gridDim.x * blockDim.x) {
    int4 v4 = reinterpret_cast<const int4*>(tets)[t];
    int v[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
    for (int s = 0; s < 6; ++s) {
      uint64_t a = (uint64_t)v[kLocalEdge[s][0]], b = (uint64_t)v[kLocalEdge[s][1]];
      uint64_t lo = a < b ? a : b, hi = a < b ? b : a;
      keys[t * 6 + s] = lo * (uint64_t)n + hi;
      vals[t * 6 + s] = (uint32_t)(t * 6 + s);
    }
  }
}

__global__ void head_flags_kernel(const uint64_t* __restrict__ keys, int64_t q,
                                  uint32_t* __restrict__ flags) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < q;
       i += (int64_t)gridDim.x * blockDim.x)
    flags[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1u : 0u;
}

// After the scan, excl[i] = number of heads before i, so the edge of item i
// is excl[i] + head(i) - 1.
__global__ void edge_emit_kernel(const uint64_t* __restrict__ keys,
                                 const uint32_t* __restrict__ vals,
                                 const uint32_t* __restrict__ excl, int64_t q,
                                 int64_t n, int32_t* __restrict__ E,
                                 int32_t* __restrict__ seg_start,
                                 int32_t* __restrict__ t2e) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < q;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t k = keys[i];
    bool head = (i == 0 || k != keys[i - 1]);
    int32_t e = (int32_t)excl[i] + (head ? 1 : 0) - 1;
    if (head) {
      E[2 * (int64_t)e] = (int32_t)(k / (uint64_t)n);
      E[2 * (int64_t)e + 1] = (int32_t)(k % (uint64_t)n);
      seg_start[e] = (int32_t)i;
    }
    t2e[vals[i]] = e;
    if (i == q - 1) seg_start[e + 1] = (int32_t)q;
  }
}

static int key_bits_for(int64_t n) {
  uint64_t maxkey = (uint64_t)n * (uint64_t)n;
  int bits = 1;
  while (bits < 64 && (maxkey >> bits) != 0) ++bits;
  return bits;
}

static unsigned grid_for(const dec_ctx* ctx, int64_t work, int threads) {
  int64_t g = (work + threads - 1) / threads;
  int64_t cap = (int64_t)ctx->num_sms * 32;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (unsigned)g;
}

dec_status build_edges(dec_ctx* ctx) {
  const int64_t q = 6 * ctx->m, n = ctx->n;
  cudaStream_t s = ctx->stream;
  DEC_TRY(ctx->key_a.ensure(q));
  DEC_TRY(ctx->key_b.ensure(q));
  DEC_TRY(ctx->val_a.ensure(q));
  DEC_TRY(ctx->val_b.ensure(q));
  DEC_TRY(ctx->flags.ensure(q));
  edge_keys_kernel<<<grid_for(ctx, ctx->m, 256), 256, 0, s>>>(
      ctx->tets.p, ctx->m, n, ctx->key_a.p, ctx->val_a.p);
  DEC_TRY(cudaGetLastError());
  ctx->launches += 1 + 1 + 3 + 1;  // keys, heads, scan, emit (sort counts itself)
  bool alt = false;
  DEC_TRY_STATUS(radix_sort_pairs(ctx, ctx->key_a.p, ctx->val_a.p, ctx->key_b.p,
                                  ctx->val_b.p, q, key_bits_for(n), &alt));
  uint64_t* keys = alt ? ctx->key_b.p : ctx->key_a.p;
  uint32_t* vals = alt ? ctx->val_b.p : ctx->val_a.p;
  head_flags_kernel<<<grid_for(ctx, q, 256), 256, 0, s>>>(keys, q, ctx->flags.p);
  DEC_TRY(cudaGetLastError());
  DEC_TRY(ctx->scan_tmp.ensure(scan_tmp_size(q)));
  DEC_TRY(exclusive_scan_u32(ctx->flags.p, ctx->flags.p, q, ctx->scan_tmp.p,
                             ctx->scan_tmp.cap, s));
  // number of edges = excl[q-1] + head(q-1)
  uint32_t last_excl = 0;
  uint64_t last_keys[2] = {0, 0};
  DEC_TRY(cudaMemcpyAsync(&last_excl, ctx->flags.p + q - 1, sizeof(uint32_t),
                          cudaMemcpyDeviceToHost, s));
  DEC_TRY(cudaMemcpyAsync(last_keys, keys + (q >= 2 ? q - 2 : 0),
                          sizeof(uint64_t) * (q >= 2 ? 2 : 1),
                          cudaMemcpyDeviceToHost, s));
  DEC_TRY(cudaStreamSynchronize(s));
  bool last_head = q < 2 || last_keys[1] != last_keys[0];
  ctx->ne = (int64_t)last_excl + (last_head ? 1 : 0);
  DEC_TRY(ctx->E.ensure(2 * ctx->ne));
  DEC_TRY(ctx->seg_start.ensure(ctx->ne + 1));
  DEC_TRY(ctx->t2e.ensure(q));
  edge_emit_kernel<<<grid_for(ctx, q, 256), 256, 0, s>>>(
      keys, vals, ctx->flags.p, q, n, ctx->E.p, ctx->seg_start.p, ctx->t2e.p);
  DEC_TRY(cudaGetLastError());
  // keep the payloads grouped by edge (tet*6+slot, increasing in each group)
  if (alt) std::swap(ctx->seg_pay, ctx->val_b);
  else std::swap(ctx->seg_pay, ctx->val_a);
  return DEC_OK;
}

// ------------------------------------------------------- CSR structure
// Row r of L holds: the lower neighbours (edges (j, r), j < r) in increasing
// j, the diagonal, then the upper neighbours (edges (r, j)) in increasing j.
// The lower lists come from the edge list sorted by (max, min).
__global__ void transpose_keys_kernel(const int32_t* __restrict__ E, int64_t ne,
                                      int64_t n, uint64_t* __restrict__ keys,
                                      uint32_t* __restrict__ vals) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne;
       e += (int64_t)gridDim.x * blockDim.x) {
    int2 ij = reinterpret_cast<const int2*>(E)[e];
    keys[e] = (uint64_t)ij.y * (uint64_t)n + (uint64_t)ij.x;
    vals[e] = (uint32_t)e;
  }
}

__global__ void row_bounds_kernel(const int32_t* __restrict__ E,
                                  const uint64_t* __restrict__ tkeys, int64_t ne,
                                  int64_t n, int32_t* __restrict__ up_begin,
                                  int32_t* __restrict__ lo_begin,
                                  int32_t* __restrict__ rowptr) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r <= n;
       r += (int64_t)gridDim.x * blockDim.x) {
    // first edge with min >= r
    int64_t lo = 0, hi = ne;
    while (lo < hi) {
      int64_t mid = (lo + hi) >> 1;
      if (E[2 * mid] < r) lo = mid + 1; else hi = mid;
    }
    int64_t ub = lo;
    // first transposed edge with max >= r
    lo = 0; hi = ne;
    const uint64_t thr = (uint64_t)r * (uint64_t)n;
    while (lo < hi) {
      int64_t mid = (lo + hi) >> 1;
      if (tkeys[mid] < thr) lo = mid + 1; else hi = mid;
    }
    up_begin[r] = (int32_t)ub;
    lo_begin[r] = (int32_t)lo;
    rowptr[r] = (int32_t)(ub + lo + r);
  }
}

__global__ void csr_fill_kernel(const int32_t* __restrict__ E,
                                const uint64_t* __restrict__ tkeys,
                                const uint32_t* __restrict__ tvals, int64_t n,
                                const int32_t* __restrict__ up_begin,
                                const int32_t* __restrict__ lo_begin,
                                const int32_t* __restrict__ rowptr,
                                int32_t* __restrict__ col, int32_t* __restrict__ eid,
                                int32_t* __restrict__ dpos,
                                int32_t* __restrict__ pos_up) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    int32_t pos = rowptr[r];
    for (int32_t k = lo_begin[r]; k < lo_begin[r + 1]; ++k) {
      col[pos] = (int32_t)(tkeys[k] % (uint64_t)n);
      eid[pos] = (int32_t)tvals[k];
      ++pos;
    }
    dpos[r] = pos;
    col[pos] = (int32_t)r;
    eid[pos] = -1;
    ++pos;
    for (int32_t e = up_begin[r]; e < up_begin[r + 1]; ++e) {
      col[pos] = E[2 * (int64_t)e + 1];
      eid[pos] = e;
      pos_up[e] = pos;
      ++pos;
    }
  }
}

dec_status build_csr_structure(dec_ctx* ctx) {
  const int64_t ne = ctx->ne, n = ctx->n;
  cudaStream_t s = ctx->stream;
  ctx->nnz = 2 * ne + n;
  if (ctx->nnz >= ((int64_t)1 << 31) - 1)
    return ctx->fail(DEC_ERR_LIMIT, "nnz of L exceeds int32 indexing");
  DEC_TRY(ctx->key_a.ensure(ne));
  DEC_TRY(ctx->key_b.ensure(ne));
  DEC_TRY(ctx->val_a.ensure(ne));
  DEC_TRY(ctx->val_b.ensure(ne));
  transpose_keys_kernel<<<grid_for(ctx, ne, 256), 256, 0, s>>>(
      ctx->E.p, ne, n, ctx->key_a.p, ctx->val_a.p);
  DEC_TRY(cudaGetLastError());
  ctx->launches += 3;  // transpose keys, row bounds, fill
  bool alt = false;
  DEC_TRY_STATUS(radix_sort_pairs(ctx, ctx->key_a.p, ctx->val_a.p, ctx->key_b.p,
                                  ctx->val_b.p, ne, key_bits_for(n), &alt));
  const uint64_t* tk = alt ? ctx->key_b.p : ctx->key_a.p;
  const uint32_t* tv = alt ? ctx->val_b.p : ctx->val_a.p;
  DEC_TRY(ctx->up_begin.ensure(n + 1));
  DEC_TRY(ctx->lo_begin.ensure(n + 1));
  DEC_TRY(ctx->rowptr.ensure(n + 1));
  DEC_TRY(ctx->col.ensure(ctx->nnz));
  DEC_TRY(ctx->eid.ensure(ctx->nnz));
  DEC_TRY(ctx->dpos.ensure(n));
  DEC_TRY(ctx->pos_up.ensure(ne));
  row_bounds_kernel<<<grid_for(ctx, n + 1, 256), 256, 0, s>>>(
      ctx->E.p, tk, ne, n, ctx->up_begin.p, ctx->lo_begin.p, ctx->rowptr.p);
  DEC_TRY(cudaGetLastError());
  csr_fill_kernel<<<grid_for(ctx, n, 128), 128, 0, s>>>(
      ctx->E.p, tk, tv, n, ctx->up_begin.p, ctx->lo_begin.p, ctx->rowptr.p,
      ctx->col.p, ctx->eid.p, ctx->dpos.p, ctx->pos_up.p);
  DEC_TRY(cudaGetLastError());
  return DEC_OK;
}

dec_status validate_mesh(dec_ctx* ctx) {
  cudaStream_t s = ctx->stream;
  DEC_TRY(ctx->errflag.ensure(4));
  DEC_TRY(cudaMemsetAsync(ctx->errflag.p, 0, sizeof(int), s));
  validate_tets_kernel<<<grid_for(ctx, ctx->m, 256), 256, 0, s>>>(
      ctx->tets.p, ctx->xyz.p, ctx->m, ctx->n, ctx->errflag.p);
  validate_tags_kernel<<<grid_for(ctx, ctx->n, 256), 256, 0, s>>>(
      ctx->tag.p, ctx->n, ctx->errflag.p);
  DEC_TRY(cudaGetLastError());
  ctx->launches += 2;
  int flag = 0;
  DEC_TRY(cudaMemcpyAsync(&flag, ctx->errflag.p, sizeof(int),
                          cudaMemcpyDeviceToHost, s));
  DEC_TRY(cudaStreamSynchronize(s));
  if (flag & 1) return ctx->fail(DEC_ERR_MESH, "a tet references a node id out of range");
  if (flag & 2) return ctx->fail(DEC_ERR_MESH, "a tet is inverted or flat (orientation <= 0)");
  if (flag & 4) return ctx->fail(DEC_ERR_MESH, "a node tag is not 0, 1 or 2");
  return DEC_OK;
}

}  // namespace dec
