// dec_api.cu - the C ABI entry points declared in include/dec.h: argument
// checks, host<->device copies and the order of the internal launches.
#include "dec_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

using dec::DevBuf;

namespace {

thread_local std::string g_create_error;

// copy `count` elements from a host or device pointer into a context buffer
template <typename T>
cudaError_t upload(DevBuf<T>& dst, const T* src, int64_t count, cudaStream_t s) {
  cudaError_t e = dst.ensure(count);
  if (e != cudaSuccess) return e;
  if (count == 0) return cudaSuccess;
  return cudaMemcpyAsync(dst.p, src, sizeof(T) * count, cudaMemcpyDefault, s);
}

template <typename T>
cudaError_t download(T* dst, const T* src, int64_t count, cudaStream_t s) {
  if (!dst || count == 0) return cudaSuccess;
  return cudaMemcpyAsync(dst, src, sizeof(T) * count, cudaMemcpyDefault, s);
}

// host copy of a host-or-device array (for argument checks of small inputs)
template <typename T>
cudaError_t host_copy(std::vector<T>& out, const T* src, int64_t count, cudaStream_t s) {
  out.resize(count);
  if (count == 0) return cudaSuccess;
  cudaError_t e = cudaMemcpyAsync(out.data(), src, sizeof(T) * count,
                                  cudaMemcpyDefault, s);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(s);
}

dec_status set_device(dec_ctx* ctx) {
  DEC_TRY(cudaSetDevice(ctx->device));
  return DEC_OK;
}

}  // namespace

extern "C" {

dec_status dec_create(dec_ctx** out, int device, void* stream) {
  if (!out) {
    g_create_error = "dec_create: ctx is NULL";
    return DEC_ERR_ARG;
  }
  *out = nullptr;
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess || device < 0 || device >= count) {
    g_create_error = std::string("dec_create: no CUDA device ") + std::to_string(device) +
                     (e != cudaSuccess ? std::string(": ") + cudaGetErrorString(e) : "");
    return e != cudaSuccess ? DEC_ERR_CUDA : DEC_ERR_ARG;
  }
  dec_ctx* ctx = new (std::nothrow) dec_ctx();
  if (!ctx) {
    g_create_error = "dec_create: out of host memory";
    return DEC_ERR_ARG;
  }
  ctx->device = device;
  e = cudaSetDevice(device);
  if (e == cudaSuccess) {
    if (stream) {
      ctx->stream = (cudaStream_t)stream;
    } else {
      e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
      ctx->own_stream = true;
    }
  }
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) {
    ctx->reduce_grid = ctx->num_sms * 8;   // the most blocks a reducing kernel runs
    e = ctx->partial.ensure((size_t)dec::kRedSlots * ctx->reduce_grid);
  }
  if (e == cudaSuccess) e = dec::init_kernel_attributes();
  if (e == cudaSuccess) e = ctx->ticket.ensure(1);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->ticket.p, 0, sizeof(unsigned), ctx->stream);
  if (e == cudaSuccess) e = ctx->cg.ensure(1);
  if (e == cudaSuccess) e = ctx->errflag.ensure(4);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    g_create_error = std::string("dec_create: ") + cudaGetErrorString(e);
    dec_destroy(ctx);
    return DEC_ERR_CUDA;
  }
  *out = ctx;
  return DEC_OK;
}

dec_status dec_destroy(dec_ctx* ctx) {
  if (!ctx) return DEC_OK;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  ctx->release_all();
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return DEC_OK;
}

const char* dec_last_error(const dec_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

dec_status dec_mesh_upload(dec_ctx* ctx, const double* xyz, int64_t n_nodes,
                           const int32_t* tets, int64_t n_tets,
                           const uint8_t* node_tag) {
  if (!ctx) return DEC_ERR_ARG;
  ctx->err.clear();
  if (!xyz || !tets || !node_tag)
    return ctx->fail(DEC_ERR_ARG, "mesh_upload: NULL pointer");
  if (n_nodes < 4 || n_nodes >= INT32_MAX)
    return ctx->fail(DEC_ERR_ARG, "mesh_upload: n_nodes must be in [4, 2^31-1)");
  if (n_tets < 1 || 6 * n_tets >= ((int64_t)1 << 32))
    return ctx->fail(DEC_ERR_ARG, "mesh_upload: n_tets must be in [1, 2^32/6)");
  DEC_TRY_STATUS(set_device(ctx));
  ctx->stage = 0;
  ctx->n = n_nodes;
  ctx->m = n_tets;
  ctx->nf = 0;              // faces of the tet-centred form: rebuilt on demand
  ctx->tet_solved = false;
  cudaStream_t s = ctx->stream;
  DEC_TRY(upload(ctx->xyz, xyz, 3 * n_nodes, s));
  DEC_TRY(upload(ctx->tets, tets, 4 * n_tets, s));
  DEC_TRY(upload(ctx->tag, node_tag, n_nodes, s));
  DEC_TRY_STATUS(dec::validate_mesh(ctx));
  DEC_TRY_STATUS(dec::build_edges(ctx));
  DEC_TRY_STATUS(dec::build_csr_structure(ctx));
  DEC_TRY_STATUS(dec::build_sell_layouts(ctx));
  ctx->grid_vec = (int)std::max<int64_t>(
      1, std::min<int64_t>((n_nodes + dec::kBlock - 1) / dec::kBlock, (int64_t)ctx->num_sms * 2));
  ctx->grid_sell = (int)std::max<int64_t>(
      1, std::min<int64_t>((ctx->sellL.nslices + 7) / 8, (int64_t)ctx->num_sms * 4));
  ctx->reduce_grid = std::max(std::max(ctx->grid_vec, ctx->grid_sell), ctx->num_sms * 8);
  DEC_TRY(ctx->partial.ensure((size_t)dec::kRedSlots * ctx->reduce_grid));
  DEC_TRY(cudaStreamSynchronize(s));
  ctx->stage = 1;
  return DEC_OK;
}

}  // extern "C"

namespace {

// Shared part of dec_hodge_assemble and dec_hodge_assemble_fields: k holds
// n_fields conductivity fields of n_tets values each (or NULL).
dec_status hodge_common(dec_ctx* ctx, const double* k, int n_fields, const double* discs,
                        int64_t n_discs, const double* scales, int32_t n_scales) {
  if (n_discs < 0 || (n_discs > 0 && !discs))
    return ctx->fail(DEC_ERR_ARG, "hodge_assemble: bad discs / n_discs");
  if (n_discs >= INT32_MAX) return ctx->fail(DEC_ERR_LIMIT, "hodge_assemble: too many discs");
  if (scales && (n_scales < 1 || n_scales > 255))
    return ctx->fail(DEC_ERR_ARG, "hodge_assemble: n_scales must be in [1, 255]");
  DEC_TRY_STATUS(set_device(ctx));
  cudaStream_t s = ctx->stream;
  ctx->stage = 1;
  // conductivity: finite and > 0
  const bool has_k = k != nullptr;
  if (has_k) {
    DEC_TRY(upload(ctx->kcond, k, (int64_t)n_fields * ctx->m, s));
    DEC_TRY_STATUS(dec::validate_k(ctx, (int64_t)n_fields * ctx->m));
  }
  std::vector<double> hs;
  if (scales) {
    DEC_TRY(host_copy(hs, scales, n_scales, s));
    for (int i = 0; i < n_scales; ++i)
      if (!(hs[i] > 0.0) || !std::isfinite(hs[i]) || (i > 0 && !(hs[i] > hs[i - 1])))
        return ctx->fail(DEC_ERR_ARG, "hodge_assemble: scales must be finite, > 0, increasing");
  } else {
    hs.assign(1, 1.0);
  }
  ctx->n_scales = (int)hs.size();
  ctx->n_fields = n_fields;
  DEC_TRY(upload(ctx->scales, hs.data(), (int64_t)hs.size(), s));
  if (n_discs > 0) {
    std::vector<double> hd;
    DEC_TRY(host_copy(hd, discs, 7 * n_discs, s));
    for (int64_t i = 0; i < n_discs; ++i) {
      const double* d = &hd[7 * i];
      bool ok = true;
      for (int j = 0; j < 7; ++j) ok = ok && std::isfinite(d[j]);
      const double nn = d[3] * d[3] + d[4] * d[4] + d[5] * d[5];
      if (!ok || !(d[6] > 0.0) || std::fabs(nn - 1.0) > 1e-9)
        return ctx->fail(DEC_ERR_ARG, "hodge_assemble: a disc needs a finite centre, unit normal and r > 0");
    }
    DEC_TRY(upload(ctx->discs, hd.data(), 7 * n_discs, s));
  }
  DEC_TRY_STATUS(dec::assemble_hodge(ctx, n_discs, has_k, n_fields));
  DEC_TRY(cudaStreamSynchronize(s));
  ctx->stage = 2;
  return DEC_OK;
}

}  // namespace

extern "C" {

dec_status dec_hodge_assemble(dec_ctx* ctx, const double* k, const double* discs,
                              int64_t n_discs, const double* scales,
                              int32_t n_scales) {
  if (!ctx) return DEC_ERR_ARG;
  ctx->err.clear();
  if (ctx->stage < 1) return ctx->fail(DEC_ERR_STATE, "hodge_assemble: no mesh uploaded");
  return hodge_common(ctx, k, 1, discs, n_discs, scales, n_scales);
}

dec_status dec_hodge_assemble_fields(dec_ctx* ctx, const double* k, int32_t n_fields,
                                     const double* discs, int64_t n_discs) {
  if (!ctx) return DEC_ERR_ARG;
  ctx->err.clear();
  if (ctx->stage < 1) return ctx->fail(DEC_ERR_STATE, "hodge_assemble_fields: no mesh uploaded");
  if (!k || n_fields < 1) return ctx->fail(DEC_ERR_ARG, "hodge_assemble_fields: bad k / n_fields");
  if (n_fields > 64)
    return ctx->fail(DEC_ERR_LIMIT, "hodge_assemble_fields: at most 64 conductivity fields");
  return hodge_common(ctx, k, n_fields, discs, n_discs, nullptr, 0);
}

dec_status dec_laplacian_build(dec_ctx* ctx, const double* T0, int32_t n_sets,
                               int32_t precond) {
  if (!ctx) return DEC_ERR_ARG;
  ctx->err.clear();
  if (ctx->stage < 2) return ctx->fail(DEC_ERR_STATE, "laplacian_build: no Hodge star assembled");
  if (!T0 || n_sets < 1) return ctx->fail(DEC_ERR_ARG, "laplacian_build: bad T0 / n_sets");
  if (precond != DEC_PRECOND_JACOBI && precond != DEC_PRECOND_FSAI &&
      precond != DEC_PRECOND_FSAI_SHARED)
    return ctx->fail(DEC_ERR_ARG, "laplacian_build: unknown preconditioner");
  if ((ctx->n_scales > 1 || ctx->n_fields > 1) && n_sets > 1)
    return ctx->fail(DEC_ERR_ARG,
                     "laplacian_build: crack states or fields and several T0 sets at once");
  DEC_TRY_STATUS(set_device(ctx));
  cudaStream_t s = ctx->stream;
  ctx->stage = 2;
  const int64_t n = ctx->n, nnz = ctx->nnz;
  ctx->n_sets = n_sets;
  ctx->precond = precond;
  ctx->B = std::max(std::max(ctx->n_scales, ctx->n_fields), n_sets);
  const bool shared = precond == DEC_PRECOND_FSAI_SHARED;
  if (shared && ctx->B > 64)
    return ctx->fail(DEC_ERR_LIMIT, "laplacian_build: a batched solve takes at most 64 instances");
  const int V = shared ? 1 : std::max(ctx->n_scales, ctx->n_fields);  // value sets
  DEC_TRY(upload(ctx->T0, T0, (int64_t)n_sets * n, s));
  DEC_TRY(ctx->val64.ensure((size_t)V * nnz));
  DEC_TRY(ctx->sL64.ensure((size_t)V * ctx->sellL.total));
  DEC_TRY(ctx->sL32.ensure((size_t)V * ctx->sellL.total));
  DEC_TRY(ctx->b.ensure((size_t)ctx->B * n));
  if (precond != DEC_PRECOND_JACOBI) {
    DEC_TRY(ctx->g64.ensure((size_t)V * nnz));
    DEC_TRY(ctx->sGlo64.ensure((size_t)V * ctx->sellLo.total));
    DEC_TRY(ctx->sGup64.ensure((size_t)V * ctx->sellUp.total));
    DEC_TRY(ctx->sGlo16.ensure((size_t)V * ctx->sellLo.total));
    DEC_TRY(ctx->sGup16.ensure((size_t)V * ctx->sellUp.total));
  } else {
    DEC_TRY(ctx->dinv64.ensure((size_t)V * n));
    DEC_TRY(ctx->dinv32.ensure((size_t)V * n));
  }
  if (shared) {
    // one shared FSAI factor (Dirichlet sets: of their common operator; crack
    // states: of the uncracked one, the fallback of the per-state factors),
    // per-entry edge data, b[n][BS]
    if (ctx->n_scales > 1) DEC_TRY_STATUS(dec::build_values_uncracked(ctx));
    else DEC_TRY_STATUS(dec::build_values(ctx, 0));
    DEC_TRY_STATUS(dec::build_precond(ctx, 0));
    DEC_TRY_STATUS(dec::batch_setup(ctx));
  } else {
    for (int inst = 0; inst < ctx->B; ++inst) DEC_TRY_STATUS(dec::build_values(ctx, inst));
    for (int vs = 0; vs < V; ++vs) DEC_TRY_STATUS(dec::build_precond(ctx, vs));
  }
  DEC_TRY(cudaStreamSynchronize(s));
  ctx->stage = 3;
  return DEC_OK;
}

dec_status dec_solve(dec_ctx* ctx, double rtol, int32_t max_iter, int32_t mode,
                     double* T_out, int32_t* iters, double* relres) {
  if (!ctx) return DEC_ERR_ARG;
  ctx->err.clear();
  if (ctx->stage < 3) return ctx->fail(DEC_ERR_STATE, "solve: no Laplacian built");
  if (!(rtol > 0.0) || !std::isfinite(rtol) || max_iter < 1)
    return ctx->fail(DEC_ERR_ARG, "solve: rtol must be > 0 and max_iter >= 1");
  if (mode != DEC_MODE_FP64 && mode != DEC_MODE_MIXED && mode != DEC_MODE_MIXED_PHASED &&
      mode != DEC_MODE_MIXED_BATCHED)
    return ctx->fail(DEC_ERR_ARG, "solve: unknown mode");
  if ((mode == DEC_MODE_MIXED_BATCHED) != (ctx->precond == DEC_PRECOND_FSAI_SHARED))
    return ctx->fail(DEC_ERR_STATE,
                     "solve: DEC_MODE_MIXED_BATCHED goes with DEC_PRECOND_FSAI_SHARED only");
  DEC_TRY_STATUS(set_device(ctx));
  cudaStream_t s = ctx->stream;
  const int64_t n = ctx->n;
  ctx->stage = 3;
  DEC_TRY(ctx->u.ensure((size_t)ctx->B * n));
  DEC_TRY(ctx->out3.ensure(3 * (size_t)ctx->B + 2));
  if (mode == DEC_MODE_FP64) {
    for (auto* bf : {&ctx->x64, &ctx->r64, &ctx->z64, &ctx->p64, &ctx->q64, &ctx->t64})
      DEC_TRY(bf->ensure(n));
  } else {
    for (auto* bf : {&ctx->x64, &ctx->r64, &ctx->t64}) DEC_TRY(bf->ensure(n));
    for (auto* bf : {&ctx->x32, &ctx->r32, &ctx->z32, &ctx->p32, &ctx->q32, &ctx->t32})
      DEC_TRY(bf->ensure(n));
  }
  ctx->iters_host.assign(ctx->B, 0);
  ctx->relres_host.assign(ctx->B, 0.0);
  dec_status worst = DEC_OK;
  if (mode == DEC_MODE_MIXED_BATCHED) {
    worst = dec::solve_batched(ctx, rtol, max_iter, ctx->iters_host.data(),
                               ctx->relres_host.data());
    if (worst == DEC_ERR_CUDA || worst == DEC_ERR_LIMIT) return worst;
  } else {
    for (int inst = 0; inst < ctx->B; ++inst) {
      dec_status st = dec::solve_instance(ctx, inst, rtol, max_iter, mode,
                                          &ctx->iters_host[inst], &ctx->relres_host[inst]);
      if (st == DEC_ERR_CUDA) return st;
      if (st != DEC_OK && worst == DEC_OK) worst = st;
    }
  }
  std::string keep = ctx->err;
  if (T_out) {
    for (int inst = 0; inst < ctx->B; ++inst) {
      DEC_TRY_STATUS(dec::form_T(ctx, inst, ctx->t64.p));
      DEC_TRY(download(T_out + (int64_t)inst * n, (const double*)ctx->t64.p, n, s));
    }
  }
  DEC_TRY(cudaStreamSynchronize(s));
  if (iters) std::copy(ctx->iters_host.begin(), ctx->iters_host.end(), iters);
  if (relres) std::copy(ctx->relres_host.begin(), ctx->relres_host.end(), relres);
  ctx->err = keep;
  ctx->stage = 4;
  return worst;
}

dec_status dec_crack_evolve(dec_ctx* ctx, int32_t rule, int32_t max_steps,
                            const int32_t* order, double rtol, int32_t max_iter, int32_t mode,
                            double k_stop, int32_t* cracked, double* k_eff, int32_t* steps) {
  if (!ctx) return DEC_ERR_ARG;
  ctx->err.clear();
  if (ctx->stage < 3) return ctx->fail(DEC_ERR_STATE, "crack_evolve: no Laplacian built");
  if (ctx->B != 1 || ctx->n_scales != 1 || ctx->precond == DEC_PRECOND_FSAI_SHARED)
    return ctx->fail(DEC_ERR_STATE,
                     "crack_evolve: needs one instance (one Dirichlet set, no crack states) "
                     "and a per-instance preconditioner");
  const int base_rule = rule & ~DEC_CRACK_REBUILD;
  if (base_rule != DEC_CRACK_MAX_FLUX && base_rule != DEC_CRACK_ORDER)
    return ctx->fail(DEC_ERR_ARG, "crack_evolve: unknown rule");
  if (mode != DEC_MODE_FP64 && mode != DEC_MODE_MIXED && mode != DEC_MODE_MIXED_PHASED)
    return ctx->fail(DEC_ERR_ARG, "crack_evolve: mode must be FP64, MIXED or MIXED_PHASED");
  if (max_steps < 0 || !cracked || !k_eff || !steps ||
      (base_rule == DEC_CRACK_ORDER && !order && max_steps > 0))
    return ctx->fail(DEC_ERR_ARG, "crack_evolve: bad max_steps or NULL output / order");
  if (!(rtol > 0.0) || !std::isfinite(rtol) || max_iter < 1 || !(k_stop >= 0.0))
    return ctx->fail(DEC_ERR_ARG, "crack_evolve: rtol > 0, max_iter >= 1, k_stop >= 0");
  DEC_TRY_STATUS(set_device(ctx));
  cudaStream_t s = ctx->stream;
  const int64_t n = ctx->n;
  std::vector<int32_t> ord;
  if (base_rule == DEC_CRACK_ORDER) DEC_TRY(host_copy(ord, order, max_steps, s));
  DEC_TRY(ctx->u.ensure((size_t)n));
  DEC_TRY(ctx->out3.ensure(5));
  if (mode == DEC_MODE_FP64) {
    for (auto* bf : {&ctx->x64, &ctx->r64, &ctx->z64, &ctx->p64, &ctx->q64, &ctx->t64})
      DEC_TRY(bf->ensure(n));
  } else {
    for (auto* bf : {&ctx->x64, &ctx->r64, &ctx->t64}) DEC_TRY(bf->ensure(n));
    for (auto* bf : {&ctx->x32, &ctx->r32, &ctx->z32, &ctx->p32, &ctx->q32, &ctx->t32})
      DEC_TRY(bf->ensure(n));
  }
  ctx->stage = 3;
  dec_status st = dec::crack_evolve(ctx, rule, max_steps, ord.data(), rtol, max_iter, mode,
                                    k_stop, cracked, k_eff, steps);
  if (st == DEC_OK) ctx->stage = 4;   // the last state's solution is current
  return st;
}

dec_status dec_set_batch_variant(dec_ctx* ctx, int32_t variant) {
  if (!ctx) return DEC_ERR_ARG;
  ctx->err.clear();
  if (variant != 0 && !dec::batch_variant_code(variant))
    return ctx->fail(DEC_ERR_ARG, "set_batch_variant: unknown variant");
  ctx->batch_force = variant;
  return DEC_OK;
}

dec_status dec_set_sell_variant(dec_ctx* ctx, int32_t l_shape, int32_t g_shape) {
  if (!ctx) return DEC_ERR_ARG;
  ctx->err.clear();
  const int vl = l_shape == 0 ? -1 : dec::sell_l_index(l_shape);
  const int vg = g_shape == 0 ? -1 : dec::sell_g_index(g_shape);
  if ((l_shape != 0 && vl < 0) || (g_shape != 0 && vg < 0))
    return ctx->fail(DEC_ERR_ARG, "set_sell_variant: unknown shape");
  ctx->sell_force_l = vl;
  ctx->sell_force_g = vg;
  // a return to the autotuner tunes again at the next solve
  if (vl < 0 || vg < 0)
    for (auto& k : ctx->sell_key) k[0] = k[1] = 0;
  return DEC_OK;
}

dec_status dec_get_sell_variant(const dec_ctx* ctx, int32_t precision, int32_t* l_shape,
                                int32_t* g_shape) {
  if (!ctx || !l_shape || !g_shape || (precision != 0 && precision != 1)) return DEC_ERR_ARG;
  *l_shape = dec::sell_l_code(ctx->sell_l[precision]);
  *g_shape = dec::sell_g_code(ctx->sell_g[precision]);
  return DEC_OK;
}

dec_status dec_get_batch_variant(dec_ctx* ctx, int32_t* gather_entries) {
  if (!ctx) return DEC_ERR_ARG;
  ctx->err.clear();
  if (!gather_entries) return ctx->fail(DEC_ERR_ARG, "get_batch_variant: NULL output");
  if (ctx->batch_variant_used < 0)
    return ctx->fail(DEC_ERR_STATE, "get_batch_variant: no batched solve yet");
  *gather_entries = ctx->batch_variant_used;
  return DEC_OK;
}

dec_status dec_k_eff(dec_ctx* ctx, double* q_in, double* q_out, double* energy) {
  if (!ctx) return DEC_ERR_ARG;
  ctx->err.clear();
  if (ctx->stage < 4) return ctx->fail(DEC_ERR_STATE, "k_eff: no solution");
  if (!q_in) return ctx->fail(DEC_ERR_ARG, "k_eff: q_in is NULL");
  DEC_TRY_STATUS(set_device(ctx));
  std::vector<double> o(3 * (size_t)ctx->B);
  DEC_TRY_STATUS(dec::k_eff_all(ctx, o.data()));
  for (int inst = 0; inst < ctx->B; ++inst) {
    q_in[inst] = o[3 * inst];
    if (q_out) q_out[inst] = o[3 * inst + 1];
    if (energy) energy[inst] = o[3 * inst + 2];
  }
  return DEC_OK;
}

dec_status dec_get_sizes(const dec_ctx* ctx, int64_t* n_nodes, int64_t* n_tets,
                         int64_t* n_edges, int64_t* nnz, int32_t* n_instances) {
  if (!ctx) return DEC_ERR_ARG;
  if (n_nodes) *n_nodes = ctx->n;
  if (n_tets) *n_tets = ctx->m;
  if (n_edges) *n_edges = ctx->ne;
  if (nnz) *nnz = ctx->nnz;
  if (n_instances) *n_instances = ctx->B;
  return DEC_OK;
}

dec_status dec_get_edges(dec_ctx* ctx, int32_t* E, int32_t* t2e) {
  if (!ctx) return DEC_ERR_ARG;
  if (ctx->stage < 1) return ctx->fail(DEC_ERR_STATE, "get_edges: no mesh");
  DEC_TRY_STATUS(set_device(ctx));
  DEC_TRY(download(E, (const int32_t*)ctx->E.p, 2 * ctx->ne, ctx->stream));
  DEC_TRY(download(t2e, (const int32_t*)ctx->t2e.p, 6 * ctx->m, ctx->stream));
  DEC_TRY(cudaStreamSynchronize(ctx->stream));
  return DEC_OK;
}

dec_status dec_get_hodge(dec_ctx* ctx, double* w, uint8_t* first_cut) {
  if (!ctx) return DEC_ERR_ARG;
  if (ctx->stage < 2) return ctx->fail(DEC_ERR_STATE, "get_hodge: no Hodge star");
  DEC_TRY_STATUS(set_device(ctx));
  DEC_TRY(download(w, (const double*)ctx->w.p, ctx->ne, ctx->stream));
  DEC_TRY(download(first_cut, (const uint8_t*)ctx->first_cut.p, ctx->ne, ctx->stream));
  DEC_TRY(cudaStreamSynchronize(ctx->stream));
  return DEC_OK;
}

dec_status dec_get_csr(dec_ctx* ctx, int32_t inst, int32_t* rowptr, int32_t* col,
                       double* val, double* b) {
  if (!ctx) return DEC_ERR_ARG;
  if (ctx->stage < 1) return ctx->fail(DEC_ERR_STATE, "get_csr: no mesh");
  if ((val || b) && ctx->stage < 3) return ctx->fail(DEC_ERR_STATE, "get_csr: no Laplacian");
  if ((val || b) && (inst < 0 || inst >= ctx->B)) return ctx->fail(DEC_ERR_ARG, "get_csr: bad instance");
  DEC_TRY_STATUS(set_device(ctx));
  cudaStream_t s = ctx->stream;
  DEC_TRY(download(rowptr, (const int32_t*)ctx->rowptr.p, ctx->n + 1, s));
  DEC_TRY(download(col, (const int32_t*)ctx->col.p, ctx->nnz, s));
  const int vs = ctx->precond != DEC_PRECOND_FSAI_SHARED ? dec::value_set(ctx, inst) : 0;
  if (val) DEC_TRY(download(val, (const double*)ctx->val64.p + (int64_t)vs * ctx->nnz, ctx->nnz, s));
  if (b) DEC_TRY(download(b, (const double*)ctx->b.p + (int64_t)inst * ctx->n, ctx->n, s));
  DEC_TRY(cudaStreamSynchronize(s));
  return DEC_OK;
}

dec_status dec_get_precond(dec_ctx* ctx, double* g) {
  if (!ctx) return DEC_ERR_ARG;
  if (ctx->stage < 3) return ctx->fail(DEC_ERR_STATE, "get_precond: no Laplacian");
  if (!g) return DEC_OK;
  DEC_TRY_STATUS(set_device(ctx));
  cudaStream_t s = ctx->stream;
  if (ctx->precond == DEC_PRECOND_FSAI) {
    DEC_TRY(download(g, (const double*)ctx->g64.p, ctx->nnz, s));
  } else {
    // Jacobi: 1/L_ii on the diagonal slots, 0 elsewhere
    std::vector<double> dinv(ctx->n);
    std::vector<int32_t> dpos(ctx->n);
    DEC_TRY(cudaMemcpyAsync(dinv.data(), ctx->dinv64.p, sizeof(double) * ctx->n,
                            cudaMemcpyDeviceToHost, s));
    DEC_TRY(cudaMemcpyAsync(dpos.data(), ctx->dpos.p, sizeof(int32_t) * ctx->n,
                            cudaMemcpyDeviceToHost, s));
    DEC_TRY(cudaStreamSynchronize(s));
    std::vector<double> full(ctx->nnz, 0.0);
    for (int64_t i = 0; i < ctx->n; ++i) full[dpos[i]] = dinv[i];
    DEC_TRY(cudaMemcpyAsync(g, full.data(), sizeof(double) * ctx->nnz, cudaMemcpyDefault, s));
  }
  DEC_TRY(cudaStreamSynchronize(s));
  return DEC_OK;
}

dec_status dec_time_kernel(dec_ctx* ctx, int32_t kernel, int32_t reps,
                           int64_t flush_bytes, double* avg_ms) {
  if (!ctx) return DEC_ERR_ARG;
  ctx->err.clear();
  if (ctx->stage < 3) return ctx->fail(DEC_ERR_STATE, "time_kernel: no Laplacian built");
  if (reps < 1 || flush_bytes < 0 || !avg_ms) return ctx->fail(DEC_ERR_ARG, "time_kernel: bad arguments");
  if ((kernel == DEC_KERNEL_FSAI_F64 || kernel == DEC_KERNEL_FSAI_BF16) &&
      ctx->precond == DEC_PRECOND_JACOBI)
    return ctx->fail(DEC_ERR_STATE, "time_kernel: no FSAI factor built");
  DEC_TRY_STATUS(set_device(ctx));
  return dec::time_kernel(ctx, kernel, reps, (size_t)flush_bytes, avg_ms);
}

dec_status dec_crack_paths(dec_ctx* ctx, int32_t n_paths, int32_t max_steps,
                           const int32_t* orders, double rtol, int32_t max_iter,
                           double k_stop, double* k_eff, int32_t* steps) {
  if (!ctx) return DEC_ERR_ARG;
  ctx->err.clear();
  if (ctx->stage < 3) return ctx->fail(DEC_ERR_STATE, "crack_paths: no Laplacian built");
  if (ctx->B != 1 || ctx->n_scales != 1 || ctx->n_fields != 1)
    return ctx->fail(DEC_ERR_STATE,
                     "crack_paths: needs one instance (one Dirichlet set, no crack states, "
                     "one conductivity field)");
  if (n_paths < 2 || n_paths > 64)
    return ctx->fail(DEC_ERR_ARG, "crack_paths: n_paths must be in [2, 64]");
  if (max_steps < 0 || (max_steps > 0 && (!orders || !k_eff)) || !steps)
    return ctx->fail(DEC_ERR_ARG, "crack_paths: bad max_steps or NULL orders / outputs");
  if (!(rtol > 0.0) || !std::isfinite(rtol) || max_iter < 1 || !(k_stop >= 0.0))
    return ctx->fail(DEC_ERR_ARG, "crack_paths: rtol > 0, max_iter >= 1, k_stop >= 0");
  DEC_TRY_STATUS(set_device(ctx));
  cudaStream_t s = ctx->stream;
  DevBuf<int32_t> ord;
  if (max_steps > 0) DEC_TRY(upload(ord, orders, (int64_t)n_paths * max_steps, s));
  ctx->stage = 3;
  dec_status st = dec::crack_paths(ctx, n_paths, max_steps, ord.p, rtol, max_iter, k_stop,
                                   k_eff, steps);
  DEC_TRY(cudaStreamSynchronize(s));
  ord.release();
  if (st == DEC_OK) ctx->stage = 4;   // the paths' last solutions are current
  return st;
}

dec_status dec_tet_solve(dec_ctx* ctx, const double* T0, double kappa, double limiter,
                         const int32_t* cracked_faces, int64_t n_cracked,
                         const double* face_flux, double rtol, int32_t max_iter, double* alpha,
                         double* q2, int32_t* iters, double* relres, int64_t* n_limited) {
  if (!ctx) return DEC_ERR_ARG;
  ctx->err.clear();
  if (ctx->stage < 1) return ctx->fail(DEC_ERR_STATE, "tet_solve: no mesh uploaded");
  if (!T0 || !(kappa > 0.0) || !std::isfinite(kappa) || !std::isfinite(limiter) ||
      n_cracked < 0 || (n_cracked > 0 && !cracked_faces))
    return ctx->fail(DEC_ERR_ARG, "tet_solve: bad T0, kappa, limiter or cracked faces");
  if (!(rtol > 0.0) || !std::isfinite(rtol) || max_iter < 1)
    return ctx->fail(DEC_ERR_ARG, "tet_solve: rtol > 0 and max_iter >= 1");
  DEC_TRY_STATUS(set_device(ctx));
  cudaStream_t s = ctx->stream;
  ctx->tet_solved = false;
  DEC_TRY_STATUS(dec::tet_faces(ctx));
  DEC_TRY(upload(ctx->tT0, T0, ctx->n, s));
  if (n_cracked > 0) DEC_TRY(upload(ctx->tcracked, cracked_faces, n_cracked, s));
  if (face_flux) DEC_TRY(upload(ctx->tflux, face_flux, ctx->nf, s));
  int it = 0;
  double rr = 0.0;
  int64_t nl = 0;
  dec_status st = dec::tet_solve(ctx, ctx->tT0.p, kappa, limiter,
                                 n_cracked > 0 ? ctx->tcracked.p : nullptr, n_cracked,
                                 face_flux ? ctx->tflux.p : nullptr, rtol, max_iter, &it, &rr,
                                 &nl);
  if (st == DEC_ERR_CUDA || st == DEC_ERR_ARG || st == DEC_ERR_LIMIT) return st;
  std::string keep = ctx->err;
  if (iters) *iters = it;
  if (relres) *relres = rr;
  if (n_limited) *n_limited = nl;
  if (alpha) DEC_TRY(download(alpha, (const double*)ctx->talpha.p, ctx->m, s));
  if (q2) DEC_TRY_STATUS(dec::tet_k_eff(ctx, q2));
  DEC_TRY(cudaStreamSynchronize(s));
  ctx->err = keep;
  ctx->tet_solved = st == DEC_OK || st == DEC_NOT_CONVERGED;
  return st;
}

dec_status dec_tet_get_faces(dec_ctx* ctx, int64_t* n_faces, int32_t* faces, int32_t* t2f) {
  if (!ctx || !n_faces) return DEC_ERR_ARG;
  ctx->err.clear();
  if (ctx->stage < 1) return ctx->fail(DEC_ERR_STATE, "tet_get_faces: no mesh uploaded");
  DEC_TRY_STATUS(set_device(ctx));
  cudaStream_t s = ctx->stream;
  DEC_TRY_STATUS(dec::tet_faces(ctx));
  *n_faces = ctx->nf;
  if (faces) DEC_TRY(download(faces, (const int32_t*)ctx->faces.p, 3 * ctx->nf, s));
  if (t2f) DEC_TRY(download(t2f, (const int32_t*)ctx->t2f.p, 4 * ctx->m, s));
  DEC_TRY(cudaStreamSynchronize(s));
  return DEC_OK;
}

dec_status dec_tet_whitney(dec_ctx* ctx, double* v) {
  if (!ctx || !v) return DEC_ERR_ARG;
  ctx->err.clear();
  if (!ctx->tet_solved) return ctx->fail(DEC_ERR_STATE, "tet_whitney: no tet-centred solution");
  DEC_TRY_STATUS(set_device(ctx));
  cudaStream_t s = ctx->stream;
  DEC_TRY(ctx->tr.ensure(3 * ctx->m));
  DEC_TRY_STATUS(dec::tet_whitney(ctx, ctx->tet_flux ? ctx->tflux.p : nullptr, ctx->tr.p));
  DEC_TRY(download(v, (const double*)ctx->tr.p, 3 * ctx->m, s));
  DEC_TRY(cudaStreamSynchronize(s));
  return DEC_OK;
}

dec_status dec_set_geom_precision(dec_ctx* ctx, int32_t precision) {
  if (!ctx) return DEC_ERR_ARG;
  ctx->err.clear();
  if (precision != DEC_GEOM_FP64 && precision != DEC_GEOM_MIXED)
    return ctx->fail(DEC_ERR_ARG, "set_geom_precision: unknown precision");
  ctx->geom_precision = precision;
  return DEC_OK;
}

dec_status dec_get_geom_fp64_tets(const dec_ctx* ctx, int64_t* n_tets) {
  if (!ctx || !n_tets) return DEC_ERR_ARG;
  *n_tets = ctx->geom_fp64_tets;
  return DEC_OK;
}

dec_status dec_get_crack_iterations(const dec_ctx* ctx, int64_t* iters) {
  if (!ctx || !iters) return DEC_ERR_ARG;
  *iters = ctx->crack_iters;
  return DEC_OK;
}

dec_status dec_get_batch_phase_ms(dec_ctx* ctx, double* ms5) {
  if (!ctx || !ms5) return DEC_ERR_ARG;
  ctx->err.clear();
  if (ctx->batch_kernel_ms < 0.0)
    return ctx->fail(DEC_ERR_STATE, "get_batch_phase_ms: no batched solve yet");
  const double it = ctx->batch_phase_ms[5] > 0.0 ? ctx->batch_phase_ms[5] : 1.0;
  for (int k = 0; k < 5; ++k) ms5[k] = ctx->batch_phase_ms[k] / it;
  return DEC_OK;
}

dec_status dec_get_batch_kernel_ms(dec_ctx* ctx, double* ms) {
  if (!ctx || !ms) return DEC_ERR_ARG;
  ctx->err.clear();
  if (ctx->batch_kernel_ms < 0.0)
    return ctx->fail(DEC_ERR_STATE, "get_batch_kernel_ms: no batched solve yet");
  *ms = ctx->batch_kernel_ms;
  return DEC_OK;
}

dec_status dec_set_barrier_test(dec_ctx* ctx, int64_t spin_limit, int32_t withhold_block) {
  if (!ctx) return DEC_ERR_ARG;
  ctx->err.clear();
  if (spin_limit < 0 || spin_limit >= (int64_t(1) << 32) || (withhold_block != 0 && withhold_block != 1))
    return ctx->fail(DEC_ERR_ARG, "set_barrier_test: spin_limit in [0, 2^32), withhold_block 0 or 1");
  ctx->test_spin_limit = (unsigned)spin_limit;
  ctx->test_withhold = (unsigned)withhold_block;
  return DEC_OK;
}

dec_status dec_get_launch_count(const dec_ctx* ctx, int64_t* count) {
  if (!ctx || !count) return DEC_ERR_ARG;
  *count = ctx->launches;
  return DEC_OK;
}

}  // extern "C"
