// dec_tet.cu - the paper's own tet-centred form (Sec. 2.3, Eq. 11-13, with
// the Sec. 3.1 Hodge limiter): one potential per tet and one flux per
// triangular face.  The flux block of Eq. 11 is diagonal ((1/kappa) *2, with
// *2_f = (dual edge length) / (face area)), so eliminating it, as the
// paper's Schur-complement solve does, leaves a two-point operator over the
// tets:
//   sum over the faces f of T of w_f (alpha_T - alpha_T'),  w_f = kappa / *2_f,
// with alpha_T' replaced by the face value T0_f (mean of the face's nodes) on
// a Dirichlet face (all three nodes Dirichlet) and the prescribed outward
// flux (Eq. 13) moved to the right-hand side on any other boundary face.
//
// The dual edge of an interior face joins the circumcentres of its two tets
// (both project onto the face's circumcentre), so its signed length is the
// sum of the two circumcentres' outward distances to the face; a boundary
// face has the one distance.  Sec. 3.1 raises *2 entries below the limiter
// to the limiter.  A cracked face (Sec. 2.5) gets w_f = 0.
//
// Faces are the sorted node triples of the tets, numbered in lexicographic
// order: key (edge id of the two smallest nodes, largest node) sorted by the
// library's radix sort.  The SPD system (at most 5 entries per row) is
// solved by FP64 PCG with an FSAI preconditioner (pattern: each tet's lower
// neighbours) in one cooperative kernel.
#include "dec_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace dec {

namespace {

constexpr int kTBlock = 256;
constexpr long kTSpinLimit = 1L << 24;

// local edge slot of the local vertex pair (a, b), a < b
__device__ __forceinline__ int pair_slot(int a, int b) {
  // (0,1) (0,2) (0,3) (1,2) (1,3) (2,3)
  return a == 0 ? b - 1 : (a == 1 ? b + 1 : 5);
}

// Face opposite local vertex v of tet t: key = (edge of its two smallest
// nodes) << 31 | largest node; payload t * 4 + v.
__global__ void face_keys_kernel(const int32_t* __restrict__ tets, const int32_t* __restrict__ t2e,
                                 int64_t m, uint64_t* __restrict__ keys,
                                 uint32_t* __restrict__ vals) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int4 v4 = reinterpret_cast<const int4*>(tets)[t];
    const int32_t g[4] = {v4.x, v4.y, v4.z, v4.w};
    for (int v = 0; v < 4; ++v) {
      int l[3], k = 0;
      for (int i = 0; i < 4; ++i)
        if (i != v) l[k++] = i;
      // sort the three local vertices by node id
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2 - i; ++j)
          if (g[l[j]] > g[l[j + 1]]) { const int x = l[j]; l[j] = l[j + 1]; l[j + 1] = x; }
      const int a = l[0] < l[1] ? l[0] : l[1], b = l[0] < l[1] ? l[1] : l[0];
      const uint32_t e = (uint32_t)t2e[t * 6 + pair_slot(a, b)];
      keys[t * 4 + v] = ((uint64_t)e << 31) | (uint64_t)(uint32_t)g[l[2]];
      vals[t * 4 + v] = (uint32_t)(t * 4 + v);
    }
  }
}

__global__ void face_heads_kernel(const uint64_t* __restrict__ keys, int64_t q,
                                  uint32_t* __restrict__ flags) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < q;
       i += (int64_t)gridDim.x * blockDim.x)
    flags[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1u : 0u;
}

// faces[f] = sorted node triple, slot0/slot1 = the owners' t*4+v (increasing
// tet id; slot1 = -1 on the boundary), t2f[t*4+v] = f
__global__ void face_fill_kernel(const uint64_t* __restrict__ keys,
                                 const uint32_t* __restrict__ vals,
                                 const uint32_t* __restrict__ excl, int64_t q,
                                 const int32_t* __restrict__ E, int32_t* __restrict__ faces,
                                 int32_t* __restrict__ slot0, int32_t* __restrict__ slot1,
                                 int32_t* __restrict__ t2f) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < q;
       i += (int64_t)gridDim.x * blockDim.x) {
    const bool head = i == 0 || keys[i] != keys[i - 1];
    const int64_t f = head ? excl[i] : excl[i] - 1;
    t2f[vals[i]] = (int32_t)f;
    if (head) {
      const uint64_t e = keys[i] >> 31;
      faces[3 * f] = E[2 * e];
      faces[3 * f + 1] = E[2 * e + 1];
      faces[3 * f + 2] = (int32_t)(keys[i] & 0x7fffffffull);
      slot0[f] = (int32_t)vals[i];
      // a boundary face (no second owner); an interior face's second entry
      // writes slot1 itself, so the head leaves it alone
      if (i + 1 == q || keys[i + 1] != keys[i]) slot1[f] = -1;
    } else {
      slot1[f] = (int32_t)vals[i];
    }
  }
}

struct D3 {
  double x, y, z;
};
__device__ __forceinline__ D3 sub(D3 a, D3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ double dot3(D3 a, D3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ D3 cross3(D3 a, D3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ D3 node(const double* xyz, int32_t i) {
  return {xyz[3 * (int64_t)i], xyz[3 * (int64_t)i + 1], xyz[3 * (int64_t)i + 2]};
}

// Per tet: outward signed distance h[t*4+v] from the circumcentre to the face
// opposite vertex v (positive when the circumcentre is inside, on the tet's
// side of the face).
__global__ void tet_heights_kernel(const double* __restrict__ xyz,
                                   const int32_t* __restrict__ tets, int64_t m,
                                   double* __restrict__ h) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int4 v4 = reinterpret_cast<const int4*>(tets)[t];
    const D3 X[4] = {node(xyz, v4.x), node(xyz, v4.y), node(xyz, v4.z), node(xyz, v4.w)};
    const D3 a = sub(X[1], X[0]), b = sub(X[2], X[0]), c = sub(X[3], X[0]);
    const D3 bxc = cross3(b, c), cxa = cross3(c, a), axb = cross3(a, b);
    const double det = dot3(a, bxc);
    const double s = 0.5 / det;
    const double aa = dot3(a, a), bb = dot3(b, b), cc = dot3(c, c);
    // circumcentre relative to X[0]
    const D3 cT = {s * (aa * bxc.x + bb * cxa.x + cc * axb.x),
                   s * (aa * bxc.y + bb * cxa.y + cc * axb.y),
                   s * (aa * bxc.z + bb * cxa.z + cc * axb.z)};
    const D3 R[4] = {{0.0, 0.0, 0.0}, a, b, c};
    for (int v = 0; v < 4; ++v) {
      const D3 p0 = R[(v + 1) & 3], p1 = R[(v + 2) & 3], p2 = R[(v + 3) & 3];
      const D3 nn = cross3(sub(p1, p0), sub(p2, p0));
      const double inv = 1.0 / sqrt(dot3(nn, nn));
      // distance of the circumcentre to the face, + towards the tet's inside
      const double dc = dot3(sub(cT, p0), nn) * inv;
      const double dv = dot3(sub(R[v], p0), nn);
      h[t * 4 + v] = dv > 0.0 ? dc : -dc;
    }
  }
}

// Per face: area, *2 = (dual edge) / area with the limiter, w = kappa / *2
// (0 when cracked), class (0 interior, 1 Dirichlet, 2 other boundary) and the
// Dirichlet face value T0_f.
__global__ void face_weights_kernel(int64_t nf, const double* __restrict__ xyz,
                                    const int32_t* __restrict__ faces,
                                    const int32_t* __restrict__ slot0,
                                    const int32_t* __restrict__ slot1,
                                    const double* __restrict__ h, const uint8_t* __restrict__ tag,
                                    const double* __restrict__ T0, const uint8_t* __restrict__ cut,
                                    double kappa, double limiter, double* __restrict__ w,
                                    uint8_t* __restrict__ cls, double* __restrict__ T0f,
                                    unsigned long long* __restrict__ n_limited) {
  unsigned long long lim = 0;
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf;
       f += (int64_t)gridDim.x * blockDim.x) {
    const int32_t a = faces[3 * f], b = faces[3 * f + 1], c = faces[3 * f + 2];
    const D3 pa = node(xyz, a), pb = node(xyz, b), pc = node(xyz, c);
    const D3 nn = cross3(sub(pb, pa), sub(pc, pa));
    const double area = 0.5 * sqrt(dot3(nn, nn));
    const int32_t s1 = slot1[f];
    const double ell = h[slot0[f]] + (s1 >= 0 ? h[s1] : 0.0);
    double star = ell / area;
    if (limiter > 0.0 && star < limiter) {
      star = limiter;
      ++lim;
    }
    w[f] = cut[f] ? 0.0 : kappa / star;
    const bool dir = s1 < 0 && tag[a] == DEC_NODE_DIRICHLET && tag[b] == DEC_NODE_DIRICHLET &&
                     tag[c] == DEC_NODE_DIRICHLET;
    cls[f] = s1 >= 0 ? 0 : (dir ? 1 : 2);
    T0f[f] = dir ? (T0[a] + T0[b] + T0[c]) / 3.0 : 0.0;
  }
  if (lim) atomicAdd(n_limited, lim);
}

__global__ void mark_cut_kernel(const int32_t* __restrict__ list, int64_t nl, int64_t nf,
                                uint8_t* __restrict__ cut, int* __restrict__ bad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nl;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t f = list[i];
    if (f < 0 || f >= nf) atomicOr(bad, 1);
    else cut[f] = 1;
  }
}

// Row T of the two-point operator in 5 slots (slot 0 the diagonal, slot
// v + 1 the neighbour across the face opposite vertex v, column -1 when
// absent or when the face carries w = 0, e.g. cracked), stored slot-major
// (k * m + T), and its right-hand side.  A tet whose faces all carry w = 0
// becomes an identity row with rhs 0.
__global__ void tet_rows_kernel(int64_t m, const int32_t* __restrict__ t2f,
                                const int32_t* __restrict__ slot0,
                                const int32_t* __restrict__ slot1, const double* __restrict__ w,
                                const uint8_t* __restrict__ cls, const double* __restrict__ T0f,
                                const double* __restrict__ flux, int32_t* __restrict__ col,
                                double* __restrict__ val, double* __restrict__ rhs) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m;
       t += (int64_t)gridDim.x * blockDim.x) {
    double d = 0.0, bt = 0.0;
    for (int v = 0; v < 4; ++v) {
      const int32_t f = t2f[t * 4 + v];
      const double wf = w[f];
      int32_t nb = -1;
      double off = 0.0;
      if (cls[f] == 0) {
        if (wf != 0.0) {
          nb = slot0[f] / 4 == (int32_t)t ? slot1[f] / 4 : slot0[f] / 4;
          off = -wf;
          d += wf;
        }
      } else if (cls[f] == 1) {
        d += wf;
        bt += wf * T0f[f];
      } else if (flux) {
        bt -= flux[f];
      }
      col[(int64_t)(v + 1) * m + t] = nb;
      val[(int64_t)(v + 1) * m + t] = off;
    }
    if (d == 0.0) {
      d = 1.0;
      bt = 0.0;
    }
    col[t] = (int32_t)t;
    val[t] = d;
    rhs[t] = bt;
  }
}

// FSAI factor of the tet operator A (the sparse-approximate-inverse family
// of the paper's ParaSails preconditioner, Sec. 2.3): row T of G has the
// pattern P = {T's lower neighbours, T}, at most 5 entries, and solves
// A[P,P] g = e_T, G_T = g / sqrt(g_T); M = G^T G.  Cholesky of the <= 5x5
// block in FP64; a pivot <= 1e-12 max(diag) (a singular block: a group of
// tets cut off by cracks) is factored again with that shift on the diagonal.
// glo[k * m + T] holds G[T][col_k(T)] for the slots k whose column is T
// (k = 0) or a lower neighbour, 0 elsewhere.
__device__ __forceinline__ double tet_entry(const int32_t* __restrict__ col,
                                            const double* __restrict__ val, int64_t m,
                                            int32_t p, int32_t q) {
  if (p == q) return val[p];
#pragma unroll
  for (int k = 1; k < 5; ++k)
    if (col[(int64_t)k * m + p] == q) return val[(int64_t)k * m + p];
  return 0.0;
}

__global__ void tet_fsai_kernel(int64_t m, const int32_t* __restrict__ col,
                                const double* __restrict__ val, double* __restrict__ glo) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m;
       t += (int64_t)gridDim.x * blockDim.x) {
    int32_t P[5];
    int slot_of[5];
    int k = 0;
    for (int s = 1; s < 5; ++s) {
      const int32_t c = col[(int64_t)s * m + t];
      if (c >= 0 && c < (int32_t)t) { P[k] = c; slot_of[k] = s; ++k; }
    }
    // ascending column order, then T itself last
    for (int i = 1; i < k; ++i)
      for (int j = i; j > 0 && P[j - 1] > P[j]; --j) {
        const int32_t c = P[j]; P[j] = P[j - 1]; P[j - 1] = c;
        const int sl = slot_of[j]; slot_of[j] = slot_of[j - 1]; slot_of[j - 1] = sl;
      }
    P[k] = (int32_t)t;
    slot_of[k] = 0;
    const int n = k + 1;
    double A[5][5];
    double dmax = 0.0;
    for (int i = 0; i < n; ++i) {
      for (int j = 0; j <= i; ++j) A[i][j] = tet_entry(col, val, m, P[i], P[j]);
      dmax = fmax(dmax, A[i][i]);
    }
    const double tiny = 1e-12 * dmax;
    double Lc[5][5];
    double shift = 0.0;
    for (int attempt = 0; attempt < 2; ++attempt) {
      bool ok = true;
      for (int i = 0; i < n && ok; ++i) {
        for (int j = 0; j <= i; ++j) {
          double sum = A[i][j] + (i == j ? shift : 0.0);
          for (int l = 0; l < j; ++l) sum -= Lc[i][l] * Lc[j][l];
          if (i == j) {
            if (!(sum > tiny)) { ok = false; break; }
            Lc[i][i] = sqrt(sum);
          } else {
            Lc[i][j] = sum / Lc[j][j];
          }
        }
      }
      if (ok) break;
      shift = tiny;
      if (attempt == 1) {            // give up: the Jacobi row of the block
        for (int i = 0; i < n; ++i)
          for (int j = 0; j <= i; ++j) Lc[i][j] = i == j ? sqrt(fmax(A[i][i], tiny) + tiny) : 0.0;
      }
    }
    // L y = e_last: y = (0, .., 0, 1 / L_nn); L^T g = y; G = g L_nn
    double g[5];
    g[n - 1] = 1.0 / (Lc[n - 1][n - 1] * Lc[n - 1][n - 1]);
    for (int i = n - 2; i >= 0; --i) {
      double sum = 0.0;
      for (int l = i + 1; l < n; ++l) sum += Lc[l][i] * g[l];
      g[i] = -sum / Lc[i][i];
    }
    const double scale = Lc[n - 1][n - 1];
    for (int s = 0; s < 5; ++s) glo[(int64_t)s * m + t] = 0.0;
    for (int i = 0; i < n; ++i) glo[(int64_t)slot_of[i] * m + t] = g[i] * scale;
  }
}

// G^T in the same slots: gup[0] = G[T][T], gup[k] = G[c][T] for an upper
// neighbour c of T (found in row c's slot whose column is T).
__global__ void tet_fsai_upper_kernel(int64_t m, const int32_t* __restrict__ col,
                                      const double* __restrict__ glo,
                                      double* __restrict__ gup) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m;
       t += (int64_t)gridDim.x * blockDim.x) {
    gup[t] = glo[t];
    for (int s = 1; s < 5; ++s) {
      const int32_t c = col[(int64_t)s * m + t];
      double v = 0.0;
      if (c > (int32_t)t) {
        for (int k = 1; k < 5; ++k)
          if (col[(int64_t)k * m + c] == (int32_t)t) v = glo[(int64_t)k * m + c];
      }
      gup[(int64_t)s * m + t] = v;
    }
  }
}

// ------------------------------------------------------------------ PCG
struct TetPcgArgs {
  int64_t m;
  const int32_t* col;
  const double* val;
  const double* rhs;
  const double* glo;        // FSAI factor G (slot-major)
  const double* gup;        // G^T in the same slots
  double* tt;               // t = G r
  double *x, *r, *p, *q;
  double* partial;          // [2][2][grid]
  unsigned* bar;            // [0] arrivals, [1] generation
  int* status;              // [0] error, [1] iterations, [2] outcome
  double* result;           // [0] |b - A x|^2, [1] |b|^2
  double rtol2;
  int max_iter;
};

__device__ __forceinline__ bool tgrid_sync(unsigned* bar, int* err) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u);
    if (arrived == gridDim.x - 1) {
      bar[0] = 0u;
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const unsigned lim = *(volatile unsigned*)(bar + 2);
      const long limit = lim ? (long)lim : kTSpinLimit;
      long polls = 0;
      unsigned ns = 32;
      while (*gen == g) {
        if (++polls > limit || *(volatile int*)err) {
          atomicExch(err, 1);
          break;
        }
        __nanosleep(ns);
        if (ns < 256) ns <<= 1;
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *(volatile int*)err == 0;
}

// Sum of NV values over the grid, identical in every block (fixed order).
template <int NV>
__device__ __forceinline__ bool tgrid_sum(const double (&v)[NV], double (&tot)[NV],
                                          double* partial, int& parity, unsigned* bar,
                                          int* err) {
  __shared__ double sh[kTBlock];
  __shared__ double bc[NV];
  double* part = partial + (size_t)parity * 2 * gridDim.x;
  parity ^= 1;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    const double s = block_sum<kTBlock>(v[k], sh);
    if (threadIdx.x == 0) part[k * gridDim.x + blockIdx.x] = s;
  }
  if (!tgrid_sync(bar, err)) return false;
  if (threadIdx.x < 32) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const double t = warp0_sum_array(part + k * gridDim.x, (int)gridDim.x);
      if (threadIdx.x == 0) bc[k] = t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) tot[k] = bc[k];
  __syncthreads();
  return true;
}

__device__ __forceinline__ double ell_row(const TetPcgArgs& a, int64_t t, const double* x) {
  double y = a.val[t] * x[t];
#pragma unroll
  for (int k = 1; k < 5; ++k) {
    const int32_t c = a.col[k * a.m + t];
    if (c >= 0) y = fma(a.val[k * a.m + t], x[c], y);
  }
  return y;
}

// sum over the row's slots of G[k][T] x[col_k(T)] (slot 0: x[T])
__device__ __forceinline__ double fsai_row(const TetPcgArgs& a, const double* G, int64_t t,
                                           const double* x) {
  double y = G[t] * x[t];
#pragma unroll
  for (int k = 1; k < 5; ++k) {
    const int32_t c = a.col[k * a.m + t];
    if (c >= 0) y = fma(G[k * a.m + t], x[c], y);
  }
  return y;
}

// PCG (FSAI M = G^T G) from x = 0 until ||b - A x|| <= rtol ||b||,
// checked on the true residual; a recursive residual that has converged but
// a true one that has not restarts from the true residual.  With FSAI the
// preconditioned residual z lives in q between the update and p = z + beta p.
__global__ void __launch_bounds__(kTBlock) tet_pcg_kernel(TetPcgArgs a) {
  if (*(volatile unsigned*)(a.bar + 3) && blockIdx.x == gridDim.x - 1) return;
  const int64_t m = a.m;
  const int64_t t0 = blockIdx.x * (int64_t)kTBlock + threadIdx.x;
  const int64_t ts = (int64_t)gridDim.x * kTBlock;
  int* err = a.status;
  int parity = 0;
  double v1[1], t1[1];
  // x = 0, r = b, |b|^2
  double bb = 0.0;
  for (int64_t t = t0; t < m; t += ts) {
    const double b = a.rhs[t];
    a.x[t] = 0.0;
    a.r[t] = b;
    bb = fma(b, b, bb);
  }
  v1[0] = bb;
  if (!tgrid_sum<1>(v1, t1, a.partial, parity, a.bar, err)) return;
  const double bnorm2 = t1[0];
  const double tol2 = a.rtol2 * bnorm2;
  int it = 0, outcome = 0, restarts = 0;
  double rr_true = bnorm2;
  if (bnorm2 > 0.0) {
    for (;;) {
      // (re)start: p = z = M r, rz
      double rz = 0.0;
      for (int64_t t = t0; t < m; t += ts) a.tt[t] = fsai_row(a, a.glo, t, a.r);
      if (!tgrid_sync(a.bar, err)) return;
      for (int64_t t = t0; t < m; t += ts) {
        const double z = fsai_row(a, a.gup, t, a.tt);
        a.p[t] = z;
        rz = fma(a.r[t], z, rz);
      }
      v1[0] = rz;
      if (!tgrid_sum<1>(v1, t1, a.partial, parity, a.bar, err)) return;
      rz = t1[0];
      bool conv = false;
      while (it < a.max_iter) {
        double pq = 0.0;
        for (int64_t t = t0; t < m; t += ts) {
          const double qt = ell_row(a, t, a.p);
          a.q[t] = qt;
          pq = fma(a.p[t], qt, pq);
        }
        v1[0] = pq;
        if (!tgrid_sum<1>(v1, t1, a.partial, parity, a.bar, err)) return;
        pq = t1[0];
        if (!(pq > 0.0) || !isfinite(pq)) { outcome = 3; break; }   // breakdown
        const double alpha = rz / pq;
        double rr = 0.0;
        for (int64_t t = t0; t < m; t += ts) {
          a.x[t] = fma(alpha, a.p[t], a.x[t]);
          const double rt = fma(-alpha, a.q[t], a.r[t]);
          a.r[t] = rt;
          rr = fma(rt, rt, rr);
        }
        v1[0] = rr;
        if (!tgrid_sum<1>(v1, t1, a.partial, parity, a.bar, err)) return;
        ++it;
        if (t1[0] <= tol2) { conv = true; break; }
        // z = G^T (G r) into q, r.z
        for (int64_t t = t0; t < m; t += ts) a.tt[t] = fsai_row(a, a.glo, t, a.r);
        if (!tgrid_sync(a.bar, err)) return;
        double rzf = 0.0;
        for (int64_t t = t0; t < m; t += ts) {
          const double z = fsai_row(a, a.gup, t, a.tt);
          a.q[t] = z;
          rzf = fma(a.r[t], z, rzf);
        }
        v1[0] = rzf;
        if (!tgrid_sum<1>(v1, t1, a.partial, parity, a.bar, err)) return;
        const double beta = t1[0] / rz;
        rz = t1[0];
        for (int64_t t = t0; t < m; t += ts) a.p[t] = fma(beta, a.p[t], a.q[t]);
        if (!tgrid_sync(a.bar, err)) return;
      }
      // true residual r = b - A x
      double rt2 = 0.0;
      for (int64_t t = t0; t < m; t += ts) {
        const double rt = a.rhs[t] - ell_row(a, t, a.x);
        a.q[t] = rt;
        rt2 = fma(rt, rt, rt2);
      }
      v1[0] = rt2;
      if (!tgrid_sum<1>(v1, t1, a.partial, parity, a.bar, err)) return;
      rr_true = t1[0];
      if (outcome == 3) break;
      if (rr_true <= tol2) { outcome = 0; break; }
      if (!conv || ++restarts > 8) { outcome = 1; break; }   // max_iter or no progress
      for (int64_t t = t0; t < m; t += ts) a.r[t] = a.q[t];
      if (!tgrid_sync(a.bar, err)) return;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.status[1] = it;
    a.status[2] = outcome;
    a.result[0] = rr_true;
    a.result[1] = bnorm2;
  }
}

// q_in / q_out through the Dirichlet faces on x = 0 / x = 1 (all three nodes
// there), block partials in fixed order
__global__ void __launch_bounds__(kTBlock)
tet_keff_kernel(int64_t nf, const double* __restrict__ xyz, const int32_t* __restrict__ faces,
                const int32_t* __restrict__ slot0, const uint8_t* __restrict__ cls,
                const double* __restrict__ w, const double* __restrict__ T0f,
                const double* __restrict__ alpha, double* __restrict__ partial) {
  __shared__ double sh[kTBlock];
  double qi = 0.0, qo = 0.0;
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf;
       f += (int64_t)gridDim.x * blockDim.x) {
    if (cls[f] != 1) continue;
    const double x0 = xyz[3 * (int64_t)faces[3 * f]], x1 = xyz[3 * (int64_t)faces[3 * f + 1]],
                 x2 = xyz[3 * (int64_t)faces[3 * f + 2]];
    const double aT = alpha[slot0[f] / 4];
    if (x0 == 0.0 && x1 == 0.0 && x2 == 0.0) qi += w[f] * (T0f[f] - aT);
    else if (x0 == 1.0 && x1 == 1.0 && x2 == 1.0) qo += w[f] * (aT - T0f[f]);
  }
  const double a = block_sum<kTBlock>(qi, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = a;
  const double b = block_sum<kTBlock>(qo, sh);
  if (threadIdx.x == 0) partial[gridDim.x + blockIdx.x] = b;
}

__global__ void tet_keff_sum_kernel(int nb, const double* __restrict__ partial,
                                    double* __restrict__ out) {
  if (threadIdx.x < 32) {
    for (int k = 0; k < 2; ++k) {
      const double s = warp0_sum_array(partial + (int64_t)k * nb, nb);
      if (threadIdx.x == 0) out[k] = s;
    }
  }
}

// Flux vector at each tet's barycentre from its face fluxes (Whitney 2-form
// interpolation): v = sum_i phi_i (b - x_i) / (3 V), phi_i the outward flux
// through the face opposite vertex i.
__global__ void tet_whitney_kernel(int64_t m, const double* __restrict__ xyz,
                                   const int32_t* __restrict__ tets,
                                   const int32_t* __restrict__ t2f,
                                   const int32_t* __restrict__ slot0,
                                   const int32_t* __restrict__ slot1,
                                   const uint8_t* __restrict__ cls, const double* __restrict__ w,
                                   const double* __restrict__ T0f,
                                   const double* __restrict__ flux,
                                   const double* __restrict__ alpha, double* __restrict__ vout) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int4 v4 = reinterpret_cast<const int4*>(tets)[t];
    const D3 X[4] = {node(xyz, v4.x), node(xyz, v4.y), node(xyz, v4.z), node(xyz, v4.w)};
    const D3 e1 = sub(X[1], X[0]), e2 = sub(X[2], X[0]), e3 = sub(X[3], X[0]);
    const double V6 = dot3(e1, cross3(e2, e3));
    const D3 bc = {0.25 * (X[0].x + X[1].x + X[2].x + X[3].x),
                   0.25 * (X[0].y + X[1].y + X[2].y + X[3].y),
                   0.25 * (X[0].z + X[1].z + X[2].z + X[3].z)};
    const double aT = alpha[t];
    D3 v = {0.0, 0.0, 0.0};
    for (int i = 0; i < 4; ++i) {
      const int32_t f = t2f[t * 4 + i];
      double phi;
      if (cls[f] == 0) {
        const int32_t other = slot0[f] / 4 == (int32_t)t ? slot1[f] / 4 : slot0[f] / 4;
        phi = w[f] * (aT - alpha[other]);
      } else if (cls[f] == 1) {
        phi = w[f] * (aT - T0f[f]);
      } else {
        phi = flux ? flux[f] : 0.0;
      }
      const D3 d = sub(bc, X[i]);
      const double s = phi * 2.0 / V6;   // phi / (3 V), V = V6 / 6
      v.x = fma(s, d.x, v.x);
      v.y = fma(s, d.y, v.y);
      v.z = fma(s, d.z, v.z);
    }
    vout[3 * t] = v.x;
    vout[3 * t + 1] = v.y;
    vout[3 * t + 2] = v.z;
  }
}

unsigned tgrid(const dec_ctx* ctx, int64_t work) {
  return (unsigned)std::max<int64_t>(
      1, std::min<int64_t>((work + 255) / 256, (int64_t)ctx->num_sms * 16));
}

}  // namespace

// Faces of the uploaded mesh (built once per mesh).
dec_status tet_faces(dec_ctx* ctx) {
  if (ctx->nf > 0) return DEC_OK;
  const int64_t m = ctx->m, q = 4 * m;
  cudaStream_t s = ctx->stream;
  DEC_TRY(ctx->key_a.ensure(q));
  DEC_TRY(ctx->key_b.ensure(q));
  DEC_TRY(ctx->val_a.ensure(q));
  DEC_TRY(ctx->val_b.ensure(q));
  DEC_TRY(ctx->flags.ensure(q));
  face_keys_kernel<<<tgrid(ctx, m), 256, 0, s>>>(ctx->tets.p, ctx->t2e.p, m, ctx->key_a.p,
                                                 ctx->val_a.p);
  DEC_TRY(cudaGetLastError());
  bool alt = false;
  DEC_TRY_STATUS(radix_sort_pairs(ctx, ctx->key_a.p, ctx->val_a.p, ctx->key_b.p, ctx->val_b.p,
                                  q, 63, &alt));
  uint64_t* keys = alt ? ctx->key_b.p : ctx->key_a.p;
  uint32_t* vals = alt ? ctx->val_b.p : ctx->val_a.p;
  face_heads_kernel<<<tgrid(ctx, q), 256, 0, s>>>(keys, q, ctx->flags.p);
  DEC_TRY(cudaGetLastError());
  DEC_TRY(ctx->scan_tmp.ensure(scan_tmp_size(q)));
  DEC_TRY(exclusive_scan_u32(ctx->flags.p, ctx->flags.p, q, ctx->scan_tmp.p, ctx->scan_tmp.cap,
                             s));
  uint32_t last_excl = 0;
  uint64_t last_keys[2] = {0, 0};
  DEC_TRY(cudaMemcpyAsync(&last_excl, ctx->flags.p + q - 1, sizeof(uint32_t),
                          cudaMemcpyDeviceToHost, s));
  DEC_TRY(cudaMemcpyAsync(last_keys, keys + (q >= 2 ? q - 2 : 0),
                          sizeof(uint64_t) * (q >= 2 ? 2 : 1), cudaMemcpyDeviceToHost, s));
  DEC_TRY(cudaStreamSynchronize(s));
  const bool last_head = q < 2 || last_keys[1] != last_keys[0];
  const int64_t nf = (int64_t)last_excl + (last_head ? 1 : 0);
  DEC_TRY(ctx->faces.ensure(3 * nf));
  DEC_TRY(ctx->fslot0.ensure(nf));
  DEC_TRY(ctx->fslot1.ensure(nf));
  DEC_TRY(ctx->t2f.ensure(q));
  face_fill_kernel<<<tgrid(ctx, q), 256, 0, s>>>(keys, vals, ctx->flags.p, q, ctx->E.p,
                                                 ctx->faces.p, ctx->fslot0.p, ctx->fslot1.p,
                                                 ctx->t2f.p);
  DEC_TRY(cudaGetLastError());
  ctx->launches += 7;   // keys, heads, scan (3), fill (the sort counts itself)
  ctx->nf = nf;
  return DEC_OK;
}

dec_status tet_solve(dec_ctx* ctx, const double* T0_dev, double kappa, double limiter,
                     const int32_t* cracked_dev, int64_t n_cracked, const double* flux_dev,
                     double rtol, int max_iter, int* iters, double* relres,
                     int64_t* n_limited) {
  DEC_TRY_STATUS(tet_faces(ctx));
  const int64_t m = ctx->m, nf = ctx->nf;
  cudaStream_t s = ctx->stream;
  DEC_TRY(ctx->tet_h.ensure(4 * m));
  DEC_TRY(ctx->fw.ensure(nf));
  DEC_TRY(ctx->fT0.ensure(nf));
  DEC_TRY(ctx->fcls.ensure(nf));
  DEC_TRY(ctx->fcut.ensure(nf));
  DEC_TRY(ctx->tcol.ensure(5 * m));
  DEC_TRY(ctx->tval.ensure(5 * m));
  DEC_TRY(ctx->trhs.ensure(m));
  DEC_TRY(ctx->tglo.ensure(5 * m));
  DEC_TRY(ctx->tgup.ensure(5 * m));
  DEC_TRY(ctx->tt.ensure(m));
  DEC_TRY(ctx->talpha.ensure(m));
  DEC_TRY(ctx->tr.ensure(m));
  DEC_TRY(ctx->tp.ensure(m));
  DEC_TRY(ctx->tq.ensure(m));
  DEC_TRY(ctx->errflag.ensure(4));
  DEC_TRY(cudaMemsetAsync(ctx->fcut.p, 0, nf, s));
  DEC_TRY(cudaMemsetAsync(ctx->errflag.p, 0, 4 * sizeof(int), s));
  if (n_cracked > 0) {
    mark_cut_kernel<<<tgrid(ctx, n_cracked), 256, 0, s>>>(cracked_dev, n_cracked, nf,
                                                           ctx->fcut.p, ctx->errflag.p);
    ctx->launches += 1;
  }
  unsigned long long* lim = reinterpret_cast<unsigned long long*>(ctx->errflag.p + 2);
  tet_heights_kernel<<<tgrid(ctx, m), 256, 0, s>>>(ctx->xyz.p, ctx->tets.p, m, ctx->tet_h.p);
  face_weights_kernel<<<tgrid(ctx, nf), 256, 0, s>>>(
      nf, ctx->xyz.p, ctx->faces.p, ctx->fslot0.p, ctx->fslot1.p, ctx->tet_h.p, ctx->tag.p,
      T0_dev, ctx->fcut.p, kappa, limiter, ctx->fw.p, ctx->fcls.p, ctx->fT0.p, lim);
  tet_rows_kernel<<<tgrid(ctx, m), 256, 0, s>>>(m, ctx->t2f.p, ctx->fslot0.p, ctx->fslot1.p,
                                                ctx->fw.p, ctx->fcls.p, ctx->fT0.p, flux_dev,
                                                ctx->tcol.p, ctx->tval.p, ctx->trhs.p);
  tet_fsai_kernel<<<tgrid(ctx, m), 256, 0, s>>>(m, ctx->tcol.p, ctx->tval.p, ctx->tglo.p);
  tet_fsai_upper_kernel<<<tgrid(ctx, m), 256, 0, s>>>(m, ctx->tcol.p, ctx->tglo.p, ctx->tgup.p);
  DEC_TRY(cudaGetLastError());
  ctx->launches += 5;
  int hflag[4];
  DEC_TRY(cudaMemcpyAsync(hflag, ctx->errflag.p, sizeof(hflag), cudaMemcpyDeviceToHost, s));
  DEC_TRY(cudaStreamSynchronize(s));
  if (hflag[0]) return ctx->fail(DEC_ERR_ARG, "tet_solve: a cracked face id is out of range");
  unsigned long long nl = 0;
  std::memcpy(&nl, &hflag[2], sizeof(nl));
  *n_limited = (int64_t)nl;
  // PCG in one cooperative kernel
  int coop = 0;
  DEC_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, ctx->device));
  if (!coop) return ctx->fail(DEC_ERR_LIMIT, "tet_solve: cooperative launch unavailable");
  int per_sm = 0;
  DEC_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tet_pcg_kernel, kTBlock, 0));
  if (per_sm < 1) return ctx->fail(DEC_ERR_LIMIT, "tet_solve: cooperative launch unavailable");
  const int grid = (int)std::max<int64_t>(
      1, std::min<int64_t>((int64_t)ctx->num_sms * std::min(per_sm, 4), (m + kTBlock - 1) / kTBlock));
  DEC_TRY(ctx->partial.ensure((size_t)4 * grid));
  DEC_TRY(ctx->coop.ensure(16));
  DEC_TRY(cudaMemsetAsync(ctx->coop.p, 0, 16 * sizeof(int64_t), s));
  unsigned* bar = reinterpret_cast<unsigned*>(ctx->coop.p);
  DEC_TRY(write_barrier_test(ctx, bar));
  TetPcgArgs a{};
  a.m = m;
  a.col = ctx->tcol.p;
  a.val = ctx->tval.p;
  a.rhs = ctx->trhs.p;
  a.glo = ctx->tglo.p;
  a.gup = ctx->tgup.p;
  a.tt = ctx->tt.p;
  a.x = ctx->talpha.p;
  a.r = ctx->tr.p;
  a.p = ctx->tp.p;
  a.q = ctx->tq.p;
  a.partial = ctx->partial.p;
  a.bar = bar;
  a.status = reinterpret_cast<int*>(ctx->coop.p + 2);
  a.result = reinterpret_cast<double*>(ctx->coop.p + 8);
  a.rtol2 = rtol * rtol;
  a.max_iter = max_iter;
  void* args[] = {&a};
  DEC_TRY(cudaLaunchCooperativeKernel((const void*)tet_pcg_kernel, dim3(grid), dim3(kTBlock),
                                      args, 0, s));
  ctx->launches += 1;
  int hs[3];
  double hr[2];
  DEC_TRY(cudaMemcpyAsync(hs, a.status, sizeof(hs), cudaMemcpyDeviceToHost, s));
  DEC_TRY(cudaMemcpyAsync(hr, a.result, sizeof(hr), cudaMemcpyDeviceToHost, s));
  DEC_TRY(cudaStreamSynchronize(s));
  *iters = hs[1];
  *relres = hr[1] > 0.0 ? std::sqrt(hr[0] / hr[1]) : 0.0;
  ctx->tet_flux = flux_dev != nullptr;
  if (hs[0]) return ctx->fail(DEC_ERR_TIMEOUT, "tet_solve: a grid barrier timed out");
  if (hs[2] == 3) return ctx->fail(DEC_ERR_BREAKDOWN, "tet_solve: CG breakdown");
  if (hs[2] == 1) return ctx->fail(DEC_NOT_CONVERGED, "tet_solve: max_iter reached");
  return DEC_OK;
}

dec_status tet_k_eff(dec_ctx* ctx, double* q2) {
  cudaStream_t s = ctx->stream;
  const unsigned G = tgrid(ctx, ctx->nf);
  DEC_TRY(ctx->kpartial.ensure((size_t)2 * G + 2));
  tet_keff_kernel<<<G, kTBlock, 0, s>>>(ctx->nf, ctx->xyz.p, ctx->faces.p, ctx->fslot0.p,
                                        ctx->fcls.p, ctx->fw.p, ctx->fT0.p, ctx->talpha.p,
                                        ctx->kpartial.p);
  tet_keff_sum_kernel<<<1, 32, 0, s>>>((int)G, ctx->kpartial.p, ctx->kpartial.p + 2 * G);
  DEC_TRY(cudaGetLastError());
  ctx->launches += 2;
  DEC_TRY(cudaMemcpyAsync(q2, ctx->kpartial.p + 2 * G, 2 * sizeof(double),
                          cudaMemcpyDeviceToHost, s));
  DEC_TRY(cudaStreamSynchronize(s));
  return DEC_OK;
}

dec_status tet_whitney(dec_ctx* ctx, const double* flux_dev, double* v_dev) {
  cudaStream_t s = ctx->stream;
  tet_whitney_kernel<<<tgrid(ctx, ctx->m), 256, 0, s>>>(
      ctx->m, ctx->xyz.p, ctx->tets.p, ctx->t2f.p, ctx->fslot0.p, ctx->fslot1.p, ctx->fcls.p,
      ctx->fw.p, ctx->fT0.p, flux_dev, ctx->talpha.p, v_dev);
  DEC_TRY(cudaGetLastError());
  ctx->launches += 1;
  return DEC_OK;
}

}  // namespace dec
