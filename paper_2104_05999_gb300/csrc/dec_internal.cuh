// dec_internal.cuh - context, device buffers and shared device helpers of
// the GB300 DEC library.  Internal: not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <string>
#include <utility>
#include <vector>

#include "../../include/dec.h"

namespace dec {

// ---------------------------------------------------------------- buffers
// A growable device allocation owned by the context; `ensure` reallocates
// only when the requested size exceeds the capacity, so repeated calls on
// meshes of the same size allocate nothing.
template <typename T>
struct DevBuf {
  T* p = nullptr;
  size_t cap = 0;
  cudaError_t ensure(size_t n) {
    if (n <= cap && p) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    size_t bytes = (n ? n : 1) * sizeof(T);
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e == cudaSuccess) cap = n;
    return e;
  }
  // like ensure, but a reallocation keeps the first `keep` elements
  cudaError_t grow_keep(size_t n, size_t keep) {
    if (n <= cap && p) return cudaSuccess;
    T* q = nullptr;
    cudaError_t e = cudaMalloc(&q, (n ? n : 1) * sizeof(T));
    if (e != cudaSuccess) return e;
    if (p && keep) e = cudaMemcpy(q, p, (keep < cap ? keep : cap) * sizeof(T), cudaMemcpyDeviceToDevice);
    if (p) cudaFree(p);
    p = q;
    cap = n;
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
};

// ------------------------------------------------- device-side scalars
// Scalars of one PCG instance kept in device memory so the iteration loop
// never needs the host.  Reductions write them from the last block.
struct CgScalars {
  double rz;        // r . z
  double pq;        // p . q
  double rr;        // r . r
  double alpha, beta;
  double bnorm2;    // b . b
  double tol2;      // (rtol * ||b||)^2
  int done;         // 1 = converged or stopped: later kernels return at once
  int iters;        // iterations taken
  int breakdown;    // 1 = p.q <= 0 or not finite
  int pad;
};

// Sliced-ELLPACK layout of one matrix sharing L's CSR structure (slices of
// 32 rows, one lane per row, rows sorted by length inside 512-row windows).
struct SellLayout {
  DevBuf<int32_t> perm;   // [nslices*32] row of each (slice, lane), -1 = none
  DevBuf<int32_t> len;    // [nslices*32] row length in slot order
  DevBuf<int32_t> sptr;   // [nslices+1] first entry of each slice
  DevBuf<int32_t> col;    // [total] column of entry j of lane l: sptr[s]+32j+l
  DevBuf<int32_t> pos;    // [nnz] CSR slot -> SELL slot, -1 if absent
  int64_t nslices = 0, total = 0;
  int C = 32, R = 512;    // rows per slice, rows per window
  void release() { perm.release(); len.release(); sptr.release(); col.release(); pos.release(); }
};

constexpr int kRedSlots = 4;           // values reduced by one kernel
constexpr int kBlock = 256;            // threads per block, vector kernels

}  // namespace dec

// ----------------------------------------------------------------- context
struct dec_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int num_sms = 152;
  std::string err;
  int stage = 0;  // 0 none, 1 mesh, 2 hodge, 3 laplacian, 4 solved

  int64_t n = 0, m = 0, ne = 0, nnz = 0;
  int n_sets = 1, n_scales = 1, B = 1;
  int precond = DEC_PRECOND_JACOBI;
  int reduce_grid = 0;  // capacity (blocks) of the reduction partials
  int grid_vec = 0;     // blocks of the element-wise vector kernels
  int grid_sell = 0;    // blocks of the SELL kernels (one slice per warp)
  int64_t launches = 0;  // kernels launched so far (graph nodes included)
  // barrier test (dec_set_barrier_test): poll limit and withheld block of
  // the persistent kernels; 0 = normal operation
  unsigned test_spin_limit = 0, test_withhold = 0;

  // mesh
  dec::DevBuf<double> xyz;
  dec::DevBuf<int32_t> tets;
  dec::DevBuf<uint8_t> tag;
  dec::DevBuf<int32_t> E;          // [ne][2]
  dec::DevBuf<int32_t> t2e;        // [m][6]
  dec::DevBuf<uint32_t> seg_pay;   // [6m] tet*6+slot, grouped by edge
  dec::DevBuf<int32_t> seg_start;  // [ne+1]
  // sort / scan scratch
  dec::DevBuf<uint64_t> key_a, key_b;
  dec::DevBuf<uint32_t> val_a, val_b;
  dec::DevBuf<uint32_t> hist, scan_tmp, flags;
  dec::DevBuf<int> errflag;        // validation / limit flags
  // Hodge star
  dec::DevBuf<double> piece;       // [6m] k_T * signed dual area
  dec::DevBuf<uint8_t> slot_cut;   // [6m] first crack state per slot
  dec::DevBuf<double> w;           // [ne] uncracked *1
  dec::DevBuf<uint8_t> first_cut;  // [ne]
  dec::DevBuf<double> discs;       // [nd][7]
  dec::DevBuf<float> discs_f;      // [nd][8]: FP32 copy for the crack pre-test
  dec::DevBuf<unsigned long long> geom_count;   // tets of the last assembly done in FP64
  int geom_precision = DEC_GEOM_FP64;           // dec_set_geom_precision
  int64_t geom_fp64_tets = 0;
  dec::DevBuf<double> scales;      // [n_scales]
  dec::DevBuf<int32_t> grid_start, grid_items;
  dec::DevBuf<double> kcond;       // [m]
  // CSR of L
  dec::DevBuf<int32_t> rowptr, col, eid, dpos, up_begin, lo_begin;
  dec::DevBuf<int32_t> pos_up;     // [ne] CSR slot of (min, max)
  dec::DevBuf<int32_t> lo_col, lo_eid;  // transposed edge list
  // values of the current instance
  dec::DevBuf<double> T0;          // [n_sets][n]
  dec::DevBuf<double> val64;       // [V][nnz] CSR values per value set
  dec::DevBuf<double> b;           // [B][n]
  dec::DevBuf<double> g64;         // [V][nnz] FSAI factor (CSR layout)
  dec::DevBuf<float> dinv32;       // [B][n]
  dec::DevBuf<double> dinv64;      // [B][n]
  // solver state
  dec::DevBuf<double> x64, r64, z64, p64, q64, t64, u;  // u: [B][n] result
  dec::DevBuf<float> x32, r32, z32, p32, q32, t32, r32b, p32b;
  dec::DevBuf<double> partial;     // [kRedSlots][reduce_grid]
  dec::DevBuf<unsigned> ticket;
  dec::DevBuf<dec::CgScalars> cg;
  dec::DevBuf<double> out3;        // k_eff outputs [B][3]
  dec::DevBuf<double> kpartial;    // k_eff block partials [3B][blocks]
  dec::DevBuf<uint8_t> flush;      // L2 eviction buffer (kernel timing only)
  // solver layouts (SELL-32-512) and their value arrays, per value set
  dec::SellLayout sellL, sellLo, sellUp;
  dec::DevBuf<double> sL64, sGlo64, sGup64;
  dec::DevBuf<float> sL32;
  dec::DevBuf<__nv_bfloat16> sGlo16, sGup16;
  dec::DevBuf<int32_t> big_rows;   // FSAI rows for the warp-per-row kernel
  dec::DevBuf<int64_t> coop;       // persistent solve: barrier, status, result
  // batched solve: sliced layouts over spatial windows, per-entry data,
  // [n][BS] vectors
  int batch_kind = 0;                      // 0 Dirichlet sets, 1 crack states, 2 fields
  int batch_BS = 0;                        // instance stride of the layouts
  dec::DevBuf<int32_t> morton;             // [n] node order of the windows
  dec::DevBuf<int32_t> mrank;              // [n] position of each node in that order
  dec::SellLayout bL, bGlo, bGup;          // L (edge or CSR form), G, G^T
  dec::DevBuf<int2> bLcw;                  // (column, FP32 value bits) per L entry
  dec::DevBuf<uint8_t> bLfc;               // first crack state per L entry (states)
  dec::DevBuf<float> bLw;                  // [total][BS] *1 per instance (fields)
  dec::DevBuf<double> bL64;                // FP64 values, [total] or [total][BS]
  dec::DevBuf<float> bd32;                 // [n] diagonal (Dirichlet sets)
  dec::DevBuf<double> bd64;
  dec::DevBuf<__nv_bfloat16> bGlo16, bGup16;   // shared factor halves
  dec::DevBuf<__nv_bfloat16> bGloB, bGupB;     // per-instance halves [total][BS]
  dec::DevBuf<__nv_bfloat16> bgb;          // per-instance factors, CSR order [nnz][BS]
  dec::DevBuf<double> bb, bx64, br64, bpartial;
  dec::DevBuf<int64_t> crack_buf;          // crack growth: block bests, picked edge
  int batch_variant[4] = {0, 0, 0, 0};     // tuned variant + 1 per stride 8..64
  int64_t batch_tune_key[4][2] = {};       // (n, nnz) each choice was tuned for
  int batch_variant_used = -1;             // variant of the last batched solve
  int batch_force = 0;                     // dec_set_batch_variant (0: autotune)
  // launch shapes of the single-instance SELL kernels per precision
  // (0: FP64, 1: FP32), tuned per (n, nnz), or forced (>= 0)
  int sell_l[2] = {-1, -1}, sell_g[2] = {-1, -1};
  int64_t sell_key[2][2] = {};
  int sell_force_l = -1, sell_force_g = -1;
  double batch_kernel_ms = -1.0;           // device time of its persistent launch
  double batch_phase_ms[6] = {};           // its per-phase times and FP32 iterations
  int64_t crack_iters = 0;                 // CG iterations of the last crack growth
  bool batch_per_instance = false;         // per-instance FSAI factors
  dec::DevBuf<float> bx, br, bz, bp, bq, bt;
  // conductivity fields (dec_hodge_assemble_fields): instances with their
  // own *1; w then holds [n_fields][ne]
  int n_fields = 1;
  // the tet-centred form (dec_tet_solve): faces, face data, the tet system
  int64_t nf = 0;                          // faces of the mesh (0: not built)
  bool tet_solved = false;
  bool tet_flux = false;                   // the last solve had face fluxes
  dec::DevBuf<int32_t> faces, fslot0, fslot1, t2f;
  dec::DevBuf<double> tet_h, fw, fT0, tval, trhs, talpha, tr, tp, tq, tT0, tflux;
  dec::DevBuf<double> tglo, tgup, tt;      // FSAI factor of the tet operator (slot-major), t
  dec::DevBuf<uint8_t> fcls, fcut;
  dec::DevBuf<int32_t> tcol, tcracked;
  std::vector<int> iters_host;
  std::vector<double> relres_host;

  void release_all() {
    xyz.release(); tets.release(); tag.release(); E.release(); t2e.release();
    seg_pay.release(); seg_start.release(); key_a.release(); key_b.release();
    val_a.release(); val_b.release(); hist.release(); scan_tmp.release();
    flags.release(); errflag.release(); piece.release(); slot_cut.release();
    w.release(); first_cut.release(); discs.release(); discs_f.release(); geom_count.release(); scales.release();
    grid_start.release(); grid_items.release(); kcond.release(); rowptr.release();
    col.release(); eid.release(); dpos.release(); up_begin.release();
    lo_begin.release(); pos_up.release(); lo_col.release(); lo_eid.release();
    T0.release(); val64.release(); b.release(); g64.release();
    dinv32.release(); dinv64.release(); x64.release();
    r64.release(); z64.release(); p64.release(); q64.release(); t64.release();
    u.release(); x32.release(); r32.release(); z32.release(); p32.release();
    q32.release(); t32.release(); r32b.release(); p32b.release(); partial.release(); ticket.release();
    cg.release(); out3.release(); flush.release();
    sellL.release(); sellLo.release(); sellUp.release(); sL64.release();
    sGlo64.release(); sGup64.release(); sL32.release(); sGlo16.release();
    sGup16.release(); big_rows.release(); coop.release();
    morton.release(); mrank.release(); bL.release(); bGlo.release(); bGup.release(); bLcw.release();
    bLfc.release(); bLw.release(); bL64.release(); bd32.release(); bd64.release();
    bGlo16.release(); bGup16.release(); bGloB.release(); bGupB.release(); bgb.release();
    bb.release(); bx64.release(); br64.release(); bpartial.release();
    kpartial.release(); crack_buf.release(); bx.release(); br.release(); bz.release();
    bp.release(); bq.release(); bt.release();
    faces.release(); fslot0.release(); fslot1.release(); t2f.release(); tet_h.release();
    fw.release(); fT0.release(); tval.release(); trhs.release();
    tglo.release(); tgup.release(); tt.release();
    talpha.release(); tr.release(); tp.release(); tq.release(); tT0.release(); tflux.release();
    fcls.release(); fcut.release(); tcol.release(); tcracked.release();
  }

  dec_status fail(dec_status s, const std::string& what) {
    err = what;
    return s;
  }
  dec_status cuda_fail(cudaError_t e, const char* what) {
    err = std::string(what) + ": " + cudaGetErrorString(e);
    return DEC_ERR_CUDA;
  }
};

#define DEC_TRY(expr)                                       \
  do {                                                      \
    cudaError_t e__ = (expr);                               \
    if (e__ != cudaSuccess) return ctx->cuda_fail(e__, #expr); \
  } while (0)

#define DEC_TRY_STATUS(expr)               \
  do {                                     \
    dec_status s__ = (expr);               \
    if (s__ != DEC_OK) return s__;         \
  } while (0)

namespace dec {

// Operator (value set) of instance `inst`: crack states and conductivity
// fields each have their own L; Dirichlet value sets share one.
inline int value_set(const dec_ctx* ctx, int inst) {
  return (ctx->n_scales > 1 || ctx->n_fields > 1) ? inst : 0;
}

// Words 2 and 3 of a persistent kernel's barrier: the poll limit of every
// wait (0 = the default) and whether the last block leaves at once.  Written
// after the barrier is cleared and before the launch, only when the
// context's barrier test is on.
inline cudaError_t write_barrier_test(dec_ctx* ctx, unsigned* bar) {
  if (!ctx->test_spin_limit && !ctx->test_withhold) return cudaSuccess;
  const unsigned v[2] = {ctx->test_spin_limit, ctx->test_withhold};
  return cudaMemcpyAsync(bar + 2, v, sizeof(v), cudaMemcpyHostToDevice, ctx->stream);
}

// ------------------------------------------------------ device helpers
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum `v` over the block into thread 0, in a fixed order (deterministic).
// GB300's FP64 pipe is narrow and a warp-wide FP64 shuffle sum costs 5 FP64
// instructions per warp, so only warp 0 adds in FP64: the block's values go
// through shared memory (sh: NT doubles) and warp 0 sums NT/32 of them per
// lane before one shuffle sum.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  sh[threadIdx.x] = v;
  __syncthreads();
  double t = 0.0;
  if (wid == 0) {
#pragma unroll
    for (int j = 0; j < NT / 32; ++j) t += sh[lane + 32 * j];
    t = warp_sum(t);
  }
  return t;
}

// The same for FP32 contributions: warps add in FP32, warp 0 adds the warp
// sums in FP64.  sh needs 32 doubles.
template <int NT>
__device__ __forceinline__ double block_sum_f(float v, double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[wid] = (double)v;
  __syncthreads();
  double t = 0.0;
  if (wid == 0) {
    t = lane < NT / 32 ? sh[lane] : 0.0;
    t = warp_sum(t);
  }
  return t;
}

// Sum of `count` doubles at p (stride 1) by warp 0, in a fixed order; the
// result is valid in lane 0 of warp 0.
__device__ __forceinline__ double warp0_sum_array(const double* p, int count) {
  double a = 0.0;
  for (int i = threadIdx.x; i < count; i += 32) a += __ldcg(p + i);
  return warp_sum(a);
}

// Deterministic grid reduction of NV doubles per thread.  Every block
// stores its block sums in partial[slot * gridDim.x + block]; the last block
// to arrive (integer ticket) sums the partials in block order and returns
// true with the totals in `tot` (valid in all its threads).  Blocks that are
// not last return false.
template <int NT, int NV>
__device__ __forceinline__ bool grid_reduce(const double (&v)[NV],
                                            double (&tot)[NV],
                                            double* partial,
                                            unsigned* ticket) {
  __shared__ double sh[NT];
  __shared__ double res[NV];
  __shared__ bool last;
#pragma unroll
  for (int s = 0; s < NV; ++s) {
    double t = block_sum<NT>(v[s], sh);
    if (threadIdx.x == 0) partial[s * gridDim.x + blockIdx.x] = t;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned k = atomicAdd(ticket, 1u);
    last = (k == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  if (threadIdx.x < 32) {
#pragma unroll
    for (int s = 0; s < NV; ++s) {
      const double t = warp0_sum_array(partial + s * gridDim.x, (int)gridDim.x);
      if (threadIdx.x == 0) res[s] = t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int s = 0; s < NV; ++s) tot[s] = res[s];
  if (threadIdx.x == 0) *ticket = 0u;
  return true;
}

}  // namespace dec

// ------------------------------------------------------ internal launches
// (defined in the .cu files; all enqueue on ctx->stream)
namespace dec {
// scan / sort
cudaError_t exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n,
                               uint32_t* tmp, size_t tmp_cap, cudaStream_t s);
size_t scan_tmp_size(int64_t n);
dec_status radix_sort_pairs(dec_ctx* ctx, uint64_t* keys, uint32_t* vals,
                            uint64_t* keys_alt, uint32_t* vals_alt, int64_t n,
                            int key_bits, bool* result_in_alt);
// mesh
dec_status validate_mesh(dec_ctx* ctx);
dec_status build_edges(dec_ctx* ctx);
dec_status build_csr_structure(dec_ctx* ctx);
dec_status build_sell_layouts(dec_ctx* ctx);
dec_status build_sell(dec_ctx* ctx, int kind, SellLayout& L, int C, int R,
                      const int32_t* order);
template <typename T>
dec_status scatter_values(dec_ctx* ctx, const SellLayout& L, const double* csr_val, T* out);
// Hodge
dec_status assemble_hodge(dec_ctx* ctx, int64_t n_discs, bool has_k, int n_fields);
dec_status validate_k(dec_ctx* ctx, int64_t count);
// system
dec_status build_values(dec_ctx* ctx, int inst);
dec_status build_precond(dec_ctx* ctx, int vs);
dec_status build_values_uncracked(dec_ctx* ctx);
// rows and FSAI rows of L changed by cracking edge e (first_cut[e] already 0)
dec_status crack_update(dec_ctx* ctx, int64_t e);
// solve
// warm: start from the current solution u of the instance instead of 0
dec_status solve_instance(dec_ctx* ctx, int inst, double rtol, int max_iter,
                          int mode, int* iters, double* relres, bool warm = false);
dec_status k_eff_all(dec_ctx* ctx, double* out3_host);   // [B][3], one pass
dec_status form_T(dec_ctx* ctx, int inst, double* T);
dec_status solve_mixed_persistent(dec_ctx* ctx, int inst, double rtol, int max_iter,
                                  int* iters_out, double* relres_out);
dec_status batch_setup(dec_ctx* ctx);
// warm: start every instance from the last batched solution
dec_status solve_batched(dec_ctx* ctx, double rtol, int max_iter, int* iters,
                         double* relres, bool warm = false);
// per-instance values of the batched layouts after per-instance *1 changed
dec_status batch_refresh_values(dec_ctx* ctx);
dec_status time_kernel(dec_ctx* ctx, int which, int reps, size_t flush_bytes,
                       double* avg_ms);
// shared-memory limits of the staged SELL kernels (current device)
cudaError_t init_kernel_attributes();
// crack growth
// the tet-centred form
int sell_l_code(int v);
int sell_g_code(int v);
int sell_l_index(int code);
int sell_g_index(int code);
bool batch_variant_code(int code);
dec_status tet_faces(dec_ctx* ctx);
dec_status tet_solve(dec_ctx* ctx, const double* T0_dev, double kappa, double limiter,
                     const int32_t* cracked_dev, int64_t n_cracked, const double* flux_dev,
                     double rtol, int max_iter, int* iters, double* relres,
                     int64_t* n_limited);
dec_status tet_k_eff(dec_ctx* ctx, double* q2);
dec_status tet_whitney(dec_ctx* ctx, const double* flux_dev, double* v_dev);
dec_status crack_paths(dec_ctx* ctx, int P, int max_steps, const int32_t* orders_dev,
                       double rtol, int max_iter, double k_stop, double* k_eff,
                       int32_t* steps);
dec_status crack_evolve(dec_ctx* ctx, int rule, int max_steps, const int32_t* order_host,
                        double rtol, int max_iter, int mode, double k_stop, int32_t* cracked,
                        double* k_eff, int32_t* steps);
}  // namespace dec
