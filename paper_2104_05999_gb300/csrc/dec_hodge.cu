// dec_hodge.cu - the diagonal Hodge star *1 on primal edges from the
// circumcentric dual (Sec. 2.1: ratio of dual to primal volumes), times the
// conductivity of the dual face (Sec. 2.1), with penny cracks making cut dual
// faces insulating (Sec. 2.5).  A per-tet conductivity k_T is carried onto
// the dual face of e as the mean of k_T over the tets around e, weighted by
// the unsigned areas of their parts of the face.
//
// One thread per tet computes, in FP64, for each of its 6 edges the signed
// area of the dual-face piece inside the tet divided by the edge length.
// The piece of edge e = (a, b) splits into two right triangles (m_e, c_F,
// c_T), one per face F = {a, b, c} of the tet containing e: legs h1 = signed
// distance from the midpoint m_e to c_F inside F (+ towards c) and h2 =
// signed distance from c_T to the plane of F (+ towards the fourth vertex).
// With h1 = |e|/2 cot(angle at c), cot = (x_a-x_c).(x_b-x_c) / |N_F| and
// h2 = (c_T - x_a).N_F / |N_F| (N_F the inward face normal, |N_F| = twice
// the face area), each half contributes
//   (1/2) h1 h2 / |e| = (1/4) (x_a-x_c).(x_b-x_c) (c_T - x_a).N_F / |N_F|^2,
// so the kernel needs one division per face and none per edge (FP64
// division and square root are expensive on GB300).  The crack test runs on
// the sub-triangles themselves, with face circumcentres computed only when
// discs are present.  A second pass sums the
// pieces of every edge (and, with a conductivity field, the k-weighted and
// plain unsigned part areas) in a fixed order (sorted tet*6+slot), so *1 is
// deterministic without atomics.
#include "dec_internal.cuh"

#include <math_constants.h>

#include <algorithm>
#include <cmath>
#include <vector>

namespace dec {

template <typename T>
struct Vec3 {
  T x, y, z;
};
using V3 = Vec3<double>;
using F3 = Vec3<float>;
__device__ __forceinline__ V3 mk(double x, double y, double z) { return {x, y, z}; }
template <typename T>
__device__ __forceinline__ Vec3<T> operator+(Vec3<T> a, Vec3<T> b) {
  return {a.x + b.x, a.y + b.y, a.z + b.z};
}
template <typename T>
__device__ __forceinline__ Vec3<T> operator-(Vec3<T> a, Vec3<T> b) {
  return {a.x - b.x, a.y - b.y, a.z - b.z};
}
template <typename T>
__device__ __forceinline__ Vec3<T> operator*(T s, Vec3<T> a) {
  return {s * a.x, s * a.y, s * a.z};
}
template <typename T>
__device__ __forceinline__ T dot(Vec3<T> a, Vec3<T> b) {
  return a.x * b.x + a.y * b.y + a.z * b.z;
}
template <typename T>
__device__ __forceinline__ Vec3<T> cross(Vec3<T> a, Vec3<T> b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

// Tet circumcentre relative to vertex 0, from the edge vectors R[1..3]:
// (|a|^2 (b x c) + |b|^2 (c x a) + |c|^2 (a x b)) / (2 a.(b x c))
template <typename T>
__device__ __forceinline__ Vec3<T> tet_circumcentre(const Vec3<T> (&R)[4]) {
  const Vec3<T> bxc = cross(R[2], R[3]), cxa = cross(R[3], R[1]), axb = cross(R[1], R[2]);
  const T det6 = dot(R[1], bxc);
  return (T(0.5) / det6) * (dot(R[1], R[1]) * bxc + dot(R[2], R[2]) * cxa +
                            dot(R[3], R[3]) * axb);
}

// circumcentre of triangle (p, p+a, p+b): p + ((|a|^2 b - |b|^2 a) x (a x b)) / (2 |a x b|^2)
__device__ __forceinline__ V3 tri_circumcentre(V3 p, V3 q, V3 r) {
  V3 a = q - p, b = r - p;
  V3 axb = cross(a, b);
  V3 num = cross(dot(a, a) * b - dot(b, b) * a, axb);
  return p + (0.5 / dot(axb, axb)) * num;
}

// Distance, in the disc's plane, from the disc centre to the segment where
// the plane meets the closed triangle (P0, P1, P2); +inf when the plane misses
// the triangle or contains it.
// s0..s2 are the signed distances dot(P_i - c, nrm) of the three points.
// Not inlined: the exact test runs for few (tet, disc) pairs, and twelve
// inlined copies made the kernel large enough to stall on instruction fetch.
__device__ __noinline__ double crack_rho_s(V3 P0, V3 P1, V3 P2, double s0, double s1,
                                           double s2, V3 c) {
  V3 P[3] = {P0, P1, P2};
  const double s[3] = {s0, s1, s2};
  int count = 0;
  V3 A = mk(0, 0, 0), B = mk(0, 0, 0);
  const int ei[3] = {0, 1, 0}, ej[3] = {1, 2, 2};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double si = s[ei[k]], sj = s[ej[k]];
    if (si * sj < 0.0) {
      double t = si / (si - sj);
      V3 X = P[ei[k]] + t * (P[ej[k]] - P[ei[k]]);
      if (count == 0) A = X; else if (count == 1) B = X;
      ++count;
    }
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if (s[i] == 0.0) {
      if (count == 0) A = P[i]; else if (count == 1) B = P[i];
      ++count;
    }
  }
  if (count == 0 || count >= 3) return CUDART_INF;
  if (count == 1) B = A;
  V3 d = B - A;
  double dd = dot(d, d);
  double tt = 0.0;
  if (dd > 0.0) tt = fmin(fmax(dot(c - A, d) / dd, 0.0), 1.0);
  V3 cl = A + tt * d;
  V3 g = c - cl;
  return sqrt(dot(g, g));
}

struct DiscGrid {
  double lo[3];
  double inv_cell;
  int dim[3];
  const int32_t* start;   // [cells+1]
  const int32_t* items;   // disc ids
  const double* discs;    // [nd][7]
  const float4* discs_f;  // [nd][2]: (centre, bound on |centre|), (normal, reach rounded up)
  const double* scales;   // [n_states]
  int n_states;
  int nd;
  double smax;            // largest radius scale
};

__constant__ int kEdgeA[6] = {0, 0, 0, 1, 1, 2};
__constant__ int kEdgeB[6] = {1, 2, 3, 2, 3, 3};
__constant__ int kEdgeC[6] = {2, 1, 1, 0, 0, 0};  // the two other vertices
__constant__ int kEdgeD[6] = {3, 3, 2, 3, 2, 1};

// The two halves of every slot's piece of dual face (below), from the edge
// vectors R[1..3] of the tet (R[0] = 0): the circumcentre cT and, per face,
// H[v] = signed distance from c_T to the face opposite v (+ towards v)
// divided by twice the face area, ((c_T - x).N) / |N|^2 with N the inward
// normal.  Half of the dual face of edge (a,b) inside face F = {a,b,c} is
// the right triangle (m_e, c_F, c_T) with legs |e|/2 * cot(angle at c) and
// the distance from c_T to F; with cot = (x_a-x_c).(x_b-x_c) / |N_F| its
// area over |e| is (1/4) (x_a-x_c).(x_b-x_c) * H_F.
template <typename T>
__device__ __forceinline__ void tet_pieces(const Vec3<T> (&R)[4], Vec3<T>& cT, T (&a0)[6],
                                           T (&a1)[6]) {
  // For a positively oriented tet the inward normals of the faces opposite
  // vertices 1, 2, 3 are the cross products the circumcentre needs, and the
  // one opposite vertex 0 is minus their sum; |N_v| is twice the face area.
  const Vec3<T> bxc = cross(R[2], R[3]), cxa = cross(R[3], R[1]), axb = cross(R[1], R[2]);
  const T det6 = dot(R[1], bxc);
  const Vec3<T> N[4] = {T(-1) * (bxc + cxa + axb), bxc, cxa, axb};
  T nn[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) nn[v] = dot(N[v], N[v]);
  // 1 / det6 and 1 / |N_v|^2: in FP64 one division of their product and
  // products of the others (the division is a long instruction sequence on
  // GB300's narrow FP64 pipe); five divisions when the product leaves the
  // normal range, and always in FP32
  T inv_det, inv_nn[4];
  bool direct = true;
  if constexpr (sizeof(T) == sizeof(double)) {
    const T p01 = det6 * nn[0], p012 = p01 * nn[1], p0123 = p012 * nn[2];
    const T prod = p0123 * nn[3];
    if (prod > 1e-280 && prod < 1e280) {
      direct = false;
      const T r = T(1) / prod;
      const T s3 = nn[3], s23 = nn[2] * s3, s123 = nn[1] * s23;
      inv_det = r * (nn[0] * s123);
      inv_nn[0] = r * (det6 * s123);
      inv_nn[1] = r * (p01 * s23);
      inv_nn[2] = r * (p012 * s3);
      inv_nn[3] = r * p0123;
    }
  }
  if (direct) {
    inv_det = T(1) / det6;
#pragma unroll
    for (int v = 0; v < 4; ++v) inv_nn[v] = T(1) / nn[v];
  }
  cT = (T(0.5) * inv_det) * (dot(R[1], R[1]) * bxc + dot(R[2], R[2]) * cxa +
                             dot(R[3], R[3]) * axb);
  // H[v]: signed distance from c_T to the face opposite v (+ towards v)
  // over twice the face area; faces 1-3 contain vertex 0 (R[0] = 0)
  T H[4];
  H[0] = dot(cT - R[1], N[0]) * inv_nn[0];
#pragma unroll
  for (int v = 1; v < 4; ++v) H[v] = dot(cT, N[v]) * inv_nn[v];
  // the six edge vectors; (x_a - x_c).(x_b - x_c) are dot products of two
  // edges at vertex c.  Slot s joins local vertices (a, b); c and d are the
  // other two (the slots of kEdgeA..D, spelled out so that every index is
  // a compile-time constant and the vectors stay in registers).
  const Vec3<T> E[4][4] = {
      {R[0], R[1], R[2], R[3]},
      {T(-1) * R[1], R[0], R[2] - R[1], R[3] - R[1]},
      {T(-1) * R[2], R[1] - R[2], R[0], R[3] - R[2]},
      {T(-1) * R[3], R[1] - R[3], R[2] - R[3], R[0]}};   // E[i][j] = x_j - x_i
  auto slot = [&](int s, int a, int b, int c, int d) {
    const T cot_c = dot(E[c][a], E[c][b]);   // face opposite d
    const T cot_d = dot(E[d][a], E[d][b]);   // face opposite c
    a0[s] = T(0.25) * cot_c * H[d];
    a1[s] = T(0.25) * cot_d * H[c];
  };
  slot(0, 0, 1, 2, 3);
  slot(1, 0, 2, 1, 3);
  slot(2, 0, 3, 1, 2);
  slot(3, 1, 2, 0, 3);
  slot(4, 1, 3, 0, 2);
  slot(5, 2, 3, 0, 1);
}

// Shape bound of the FP32 geometry (DEC_GEOM_MIXED): a tet is computed in
// FP32 when L^3 <= kShapeMax |6 V|, L the longest of its edges from vertex 0
// (a regular tet has 2.8, a Kuhn tet 5.2; 96 % of the tets of a jittered
// Delaunay cube pass 16), in FP64 otherwise.
constexpr float kShapeMax = 16.0f;

// MIXED = false: every tet in FP64.  MIXED = true: well-shaped tets in FP32.
// n_fp64 counts the tets computed in FP64.
template <bool MIXED>
__global__ void __launch_bounds__(128, 3)
hodge_tet_kernel(const double* __restrict__ xyz, const int32_t* __restrict__ tets,
                 const double* __restrict__ kcond, int64_t m,
                 double* __restrict__ piece, double* __restrict__ kpart,
                 uint8_t* __restrict__ slot_cut, DiscGrid grid,
                 unsigned long long* __restrict__ n_fp64) {
  unsigned n64 = 0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m;
       t += (int64_t)gridDim.x * blockDim.x) {
    int4 v4 = reinterpret_cast<const int4*>(tets)[t];
    const int vid[4] = {v4.x, v4.y, v4.z, v4.w};
    V3 X[4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
      X[i] = mk(xyz[3 * (int64_t)vid[i]], xyz[3 * (int64_t)vid[i] + 1],
                xyz[3 * (int64_t)vid[i] + 2]);
    const double kT = kcond ? kcond[t] : 1.0;
    const int64_t q6 = 6 * m;
    V3 cT;                 // circumcentre relative to X[0]
    double a0[6], a1[6];
    double Et = 0.0;       // bound on the error of cT (FP32 geometry)
    bool fast = false;
    if constexpr (MIXED) {
      // edge vectors formed in FP64 and rounded once: each coordinate
      // carries a relative error of at most 2^-24
      F3 Rf[4];
      Rf[0] = {0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int i = 1; i < 4; ++i)
        Rf[i] = {(float)(X[i].x - X[0].x), (float)(X[i].y - X[0].y),
                 (float)(X[i].z - X[0].z)};
      const float det6 = fabsf(dot(Rf[1], cross(Rf[2], Rf[3])));
      const float L2 = fmaxf(dot(Rf[1], Rf[1]), fmaxf(dot(Rf[2], Rf[2]), dot(Rf[3], Rf[3])));
      const float L = sqrtf(L2);
      if (L2 * L <= kShapeMax * det6) {
        fast = true;
        F3 cTf;
        float b0[6], b1[6];
        tet_pieces(Rf, cTf, b0, b1);
#pragma unroll
        for (int s = 0; s < 6; ++s) {
          a0[s] = b0[s];
          a1[s] = b1[s];
        }
        cT = mk(cTf.x, cTf.y, cTf.z);
        // With rho = L^3 / |6V| the rounded edge vectors move the
        // circumcentre (the solution of 2 R c = |R_i|^2, whose matrix has
        // smallest singular value >= |6V| / (3 L^2)) by at most
        // (17 rho + 24 rho^2) u L; the formula's own roundings are of the same
        // order.  Et doubles the sum (u = 2^-24).
        const double rho = (double)(L2 * L) / (double)det6;
        Et = 64.0 * 5.9604645e-8 * rho * (1.0 + rho) * (double)L;
      }
    }
    if (!fast) {
      V3 R[4];
      R[0] = mk(0.0, 0.0, 0.0);
#pragma unroll
      for (int i = 1; i < 4; ++i) R[i] = X[i] - X[0];
      tet_pieces(R, cT, a0, a1);
      ++n64;
    }
    uint8_t first[6];
#pragma unroll
    for (int s = 0; s < 6; ++s) {
      piece[t * 6 + s] = a0[s] + a1[s];
      if (kcond) {                       // unsigned part of the face, with and without k
        const double u = fabs(a0[s]) + fabs(a1[s]);
        kpart[t * 6 + s] = kT * u;
        kpart[q6 + t * 6 + s] = u;
      }
      first[s] = (uint8_t)grid.n_states;
    }
    if (grid.nd > 0) {
      // Every dual sub-triangle of the tet lies in its circumball (c_T is
      // the centre; m_e and c_F are projections of c_T onto an edge line and
      // a face plane), so a disc that misses the ball cuts none of them and
      // the candidate discs are those binned in the cells the ball's box
      // meets.  The radius carries a relative margin; the cut decision
      // itself stays exact.
      // With FP32 geometry the ball is centred on the rounded circumcentre
      // and its radius grows by twice the error bound, so it still holds the
      // exact ball; the exact circumcentre cTx is then formed in FP64 for a
      // tet that some disc may cut.
      const V3 cTa = X[0] + cT;
      double RT2, RT;
      if (fast) {
        RT = (sqrt(dot(cT, cT)) + 2.0 * Et) * (1.0 + 1e-9);
        RT2 = RT * RT;
      } else {
        RT2 = dot(cT, cT) * (1.0 + 1e-9) + 1e-300;
        RT = sqrt(RT2);
      }
      V3 cTx = cTa;
      bool have_cTx = !fast;
      const double lo[3] = {cTa.x - RT, cTa.y - RT, cTa.z - RT};
      const double hi[3] = {cTa.x + RT, cTa.y + RT, cTa.z + RT};
      // face circumcentres: only for a tet that some disc may cut
      V3 cF[4];
      bool have_cF = false;
      int c0[3], c1[3];
      bool empty = false;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        double f0 = (lo[d] - grid.lo[d]) * grid.inv_cell;
        double f1 = (hi[d] - grid.lo[d]) * grid.inv_cell;
        if (f1 < 0.0 || f0 >= (double)grid.dim[d]) empty = true;
        c0[d] = (int)fmax(0.0, floor(f0));
        c1[d] = (int)fmin((double)grid.dim[d] - 1.0, floor(f1));
      }
      // The ball test is conservative (the in-plane reach is bounded by
      // r + R_T).  Signed distances to the disc plane of the 11 points of
      // the 12 dual sub-triangles (6 edge midpoints, 4 face circumcentres,
      // c_T) are computed once per disc; a sub-triangle strictly on one side
      // of the plane cannot be cut and skips the exact test.
      //
      // Most candidate discs are far from the tet, and GB300's FP64 pipe is
      // narrow, so the two rejections are first made entirely in FP32 from
      // c_T rounded once per tet and the discs rounded once on the host.
      // With u = 2^-24 and S = A_t + A_d (bounds on |c_T| and |centre| per
      // coordinate), the offset v = c_T - centre carries an error of at most
      // 2uS per coordinate, so (first order, |normal| = 1):
      //   |dp32 - dp| <= 6 sqrt(3) u S,   |par32 - par| <= 63 u S^2
      // (dp the distance to the disc plane, par = |v|^2 - dp^2).  The
      // margins below are twice these plus the roundings of the thresholds,
      // so FP32 rejects only where the FP64 test rejects too: the decisions,
      // and so *1 and the crack states, are unchanged.
      constexpr float kU = 5.9604645e-8f;    // 2^-24
      const float Cx = (float)cTa.x, Cy = (float)cTa.y, Cz = (float)cTa.z;
      const float At = fmaxf(fabsf(Cx), fmaxf(fabsf(Cy), fabsf(Cz))) * (1.0f + 2.0f * kU);
      const float RTf = (float)RT * (1.0f + 4.0f * kU);
      auto test_disc = [&](int id) {
        {
          const float4 d0 = __ldg(grid.discs_f + 2 * (int64_t)id);
          const float4 d1 = __ldg(grid.discs_f + 2 * (int64_t)id + 1);
          const float vx = Cx - d0.x, vy = Cy - d0.y, vz = Cz - d0.z;
          const float S = At + d0.w;
          const float dpf = fmaf(vx, d1.x, fmaf(vy, d1.y, vz * d1.z));
          if (fabsf(dpf) > RTf + (24.0f * S + 8.0f * RTf) * kU) return;   // ball misses the plane
          const float vv = fmaf(vx, vx, fmaf(vy, vy, vz * vz));
          const float par = fmaf(-dpf, dpf, vv);
          const float T = d1.w + RTf;
          if (par > T * T * (1.0f + 8.0f * kU) + 128.0f * kU * S * S) return;   // misses the disc
        }
        const double* dsc = grid.discs + 7 * (int64_t)id;
        V3 dc = mk(dsc[0], dsc[1], dsc[2]);
        V3 dn = mk(dsc[3], dsc[4], dsc[5]);
        const double r = dsc[6];
        {
          const V3 v = cTa - dc;
          const double dp = dot(v, dn);
          if (dp * dp > RT2) return;                      // ball misses the plane
          const double par2 = dot(v, v) - dp * dp;
          const double reach = grid.smax * r * (1.0 + 1e-9);
          if (par2 > reach * reach + 2.0 * reach * RT + RT2) return;
        }
        if (!have_cF) {
#pragma unroll
          for (int v = 0; v < 4; ++v)
            cF[v] = tri_circumcentre(X[(v + 1) & 3], X[(v + 2) & 3], X[(v + 3) & 3]);
          have_cF = true;
        }
        if (!have_cTx) {
          V3 R[4];
          R[0] = mk(0.0, 0.0, 0.0);
#pragma unroll
          for (int i = 1; i < 4; ++i) R[i] = X[i] - X[0];
          cTx = X[0] + tet_circumcentre(R);
          have_cTx = true;
        }
        const double sT = dot(cTx - dc, dn);
        double sF[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) sF[v] = dot(cF[v] - dc, dn);
#pragma unroll 1
        for (int s = 0; s < 6; ++s) {
          if (first[s] == 0) continue;
          V3 me = 0.5 * (X[kEdgeA[s]] + X[kEdgeB[s]]);
          const double sM = dot(me - dc, dn);
#pragma unroll 1
          for (int h = 0; h < 2; ++h) {
            const int opp = h == 0 ? kEdgeD[s] : kEdgeC[s];
            const double sf = sF[opp];
            if ((sM > 0.0 && sf > 0.0 && sT > 0.0) || (sM < 0.0 && sf < 0.0 && sT < 0.0))
              continue;                                   // no crossing: rho = inf
            const double rho = crack_rho_s(me, cF[opp], cTx, sM, sf, sT, dc);
            for (int st = 0; st < (int)first[s]; ++st)
              if (rho <= grid.scales[st] * r) {
                first[s] = (uint8_t)st;
                break;
              }
          }
        }
      };
      if (!empty) {
        const int64_t ncell = (int64_t)(c1[0] - c0[0] + 1) * (c1[1] - c0[1] + 1) *
                              (c1[2] - c0[2] + 1);
        // a far circumcentre (flat boundary tet): fewer tests without the
        // grid, i.e. every disc once (one pass of the loops below); one call
        // site of test_disc keeps the kernel small
        const bool all = ncell > grid.nd;
        if (all) c1[0] = c0[0], c1[1] = c0[1], c1[2] = c0[2];
        for (int gz = c0[2]; gz <= c1[2]; ++gz)
          for (int gy = c0[1]; gy <= c1[1]; ++gy)
            for (int gx = c0[0]; gx <= c1[0]; ++gx) {
              const int cell = gx + grid.dim[0] * (gy + grid.dim[1] * gz);
              const int i0 = all ? 0 : grid.start[cell];
              const int i1 = all ? grid.nd : grid.start[cell + 1];
              for (int it = i0; it < i1; ++it) test_disc(all ? it : grid.items[it]);
            }
      }
    }
#pragma unroll
    for (int s = 0; s < 6; ++s) slot_cut[t * 6 + s] = first[s];
  }
  // tets computed in FP64: one atomic per warp
  const unsigned w64 = __reduce_add_sync(0xffffffffu, n64);
  if ((threadIdx.x & 31) == 0 && w64) atomicAdd(n_fp64, (unsigned long long)w64);
}

// *1[e] = sum of the pieces of e (already divided by |e|), in increasing
// tet*6+slot order, times kappa_e = sum k_T u_T / sum u_T (u_T the unsigned
// part areas, kpart = [k u | u], absent for k = 1); first_cut[e] = min over
// those slots.
__global__ void edge_reduce_kernel(const int32_t* __restrict__ seg_start,
                                   const uint32_t* __restrict__ seg_pay,
                                   const double* __restrict__ piece,
                                   const double* __restrict__ kpart, int64_t q6,
                                   const uint8_t* __restrict__ slot_cut,
                                   int64_t ne, double* __restrict__ w,
                                   uint8_t* __restrict__ first_cut) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne;
       e += (int64_t)gridDim.x * blockDim.x) {
    double sum = 0.0, ku = 0.0, u = 0.0;
    unsigned fc = 255u;
    for (int32_t k = seg_start[e]; k < seg_start[e + 1]; ++k) {
      uint32_t p = seg_pay[k];
      sum += piece[p];
      if (kpart) {
        ku += kpart[p];
        u += kpart[q6 + p];
      }
      fc = min(fc, (unsigned)slot_cut[p]);
    }
    if (kpart) sum = u > 0.0 ? sum * (ku / u) : 0.0;
    w[e] = sum;
    first_cut[e] = (uint8_t)fc;
  }
}

// *1 of conductivity fields 1..F-1 (field 0 comes from edge_reduce_kernel):
// the same fixed-order sums with k_f[t] u_T in place of k_0[t] u_T, so a
// field's *1 equals, bit for bit, what a single-field assembly with that k
// gives.
__global__ void edge_reduce_fields_kernel(const int32_t* __restrict__ seg_start,
                                          const uint32_t* __restrict__ seg_pay,
                                          const double* __restrict__ piece,
                                          const double* __restrict__ upart,
                                          const double* __restrict__ kf, int64_t m, int F,
                                          int64_t ne, double* __restrict__ w) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne;
       e += (int64_t)gridDim.x * blockDim.x) {
    double sum = 0.0, u = 0.0;
    const int32_t k0 = seg_start[e], k1 = seg_start[e + 1];
    for (int32_t k = k0; k < k1; ++k) {
      const uint32_t p = seg_pay[k];
      sum += piece[p];
      u += upart[p];
    }
    for (int f = 1; f < F; ++f) {
      const double* kk = kf + (int64_t)f * m;
      double ku = 0.0;
      for (int32_t k = k0; k < k1; ++k) {
        const uint32_t p = seg_pay[k];
        ku += __dmul_rn(kk[p / 6], upart[p]);   // the product kpart holds: no FMA
      }
      w[(int64_t)f * ne + e] = u > 0.0 ? sum * (ku / u) : 0.0;
    }
  }
}

// uniform grid of disc bounding boxes (radius scaled by the largest state)
__global__ void disc_bin_kernel(const double* __restrict__ discs, int nd,
                                double smax, DiscGrid g, int32_t* __restrict__ counts,
                                int32_t* __restrict__ cursor,
                                int32_t* __restrict__ items, int fill) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nd;
       i += gridDim.x * blockDim.x) {
    const double* d = discs + 7 * (int64_t)i;
    const double R = d[6] * smax;
    int c0[3], c1[3];
    for (int k = 0; k < 3; ++k) {
      c0[k] = max(0, (int)floor((d[k] - R - g.lo[k]) * g.inv_cell));
      c1[k] = min(g.dim[k] - 1, (int)floor((d[k] + R - g.lo[k]) * g.inv_cell));
    }
    for (int z = c0[2]; z <= c1[2]; ++z)
      for (int y = c0[1]; y <= c1[1]; ++y)
        for (int x = c0[0]; x <= c1[0]; ++x) {
          int cell = x + g.dim[0] * (y + g.dim[1] * z);
          if (!fill) atomicAdd(&counts[cell], 1);
          else items[atomicAdd(&cursor[cell], 1)] = i;
        }
  }
}

__global__ void copy_i32_kernel(const int32_t* a, int32_t* b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = a[i];
}

__global__ void validate_k_kernel(const double* __restrict__ k, int64_t m, int* errflag) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m;
       t += (int64_t)gridDim.x * blockDim.x) {
    const double v = k[t];
    if (!(v > 0.0) || !isfinite(v)) atomicOr(errflag, 16);
  }
}

// conductivity must be finite and > 0 (checked on the device)
dec_status validate_k(dec_ctx* ctx, int64_t count) {
  cudaStream_t s = ctx->stream;
  DEC_TRY(cudaMemsetAsync(ctx->errflag.p, 0, sizeof(int), s));
  const unsigned g = (unsigned)std::max<int64_t>(
      1, std::min<int64_t>((count + 255) / 256, (int64_t)ctx->num_sms * 16));
  validate_k_kernel<<<g, 256, 0, s>>>(ctx->kcond.p, count, ctx->errflag.p);
  DEC_TRY(cudaGetLastError());
  ctx->launches += 1;
  int flag = 0;
  DEC_TRY(cudaMemcpyAsync(&flag, ctx->errflag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  DEC_TRY(cudaStreamSynchronize(s));
  if (flag & 16) return ctx->fail(DEC_ERR_ARG, "hodge_assemble: conductivity must be finite and > 0");
  return DEC_OK;
}

dec_status assemble_hodge(dec_ctx* ctx, int64_t nd, bool has_k, int n_fields) {
  cudaStream_t s = ctx->stream;
  const int64_t m = ctx->m, q = 6 * m;
  DEC_TRY(ctx->piece.ensure(has_k ? 3 * q : q));   // [piece | k u | u]
  DEC_TRY(ctx->slot_cut.ensure(q));
  DEC_TRY(ctx->w.ensure((size_t)n_fields * ctx->ne));
  DEC_TRY(ctx->first_cut.ensure(ctx->ne));
  DiscGrid g{};
  g.nd = (int)nd;
  g.n_states = ctx->n_scales;
  g.discs = ctx->discs.p;
  g.scales = ctx->scales.p;
  if (nd > 0) {
    // grid bounds from a host copy of the discs
    std::vector<double> hd(7 * nd), hs(ctx->n_scales);
    DEC_TRY(cudaMemcpyAsync(hd.data(), ctx->discs.p, sizeof(double) * 7 * nd,
                            cudaMemcpyDeviceToHost, s));
    DEC_TRY(cudaMemcpyAsync(hs.data(), ctx->scales.p, sizeof(double) * ctx->n_scales,
                            cudaMemcpyDeviceToHost, s));
    DEC_TRY(cudaStreamSynchronize(s));
    const double smax = hs.back();
    g.smax = smax;
    // FP32 disc records for the pre-test: centre and a bound on its largest
    // coordinate, normal and the reach smax * r (1 + 1e-9), bounds rounded up
    std::vector<float> hf(8 * nd);
    constexpr double kUp = 1.0 + 2.4e-7;     // 1 + 4 * 2^-24
    for (int64_t i = 0; i < nd; ++i) {
      const double* d = hd.data() + 7 * i;
      float* f = hf.data() + 8 * i;
      double amax = 0.0;
      for (int k = 0; k < 3; ++k) {
        f[k] = (float)d[k];
        f[4 + k] = (float)d[3 + k];
        amax = std::max(amax, std::fabs(d[k]));
      }
      f[3] = (float)(amax * kUp);
      f[7] = (float)(smax * d[6] * (1.0 + 1e-9) * kUp);
    }
    DEC_TRY(ctx->discs_f.ensure(8 * nd));
    DEC_TRY(cudaMemcpyAsync(ctx->discs_f.p, hf.data(), sizeof(float) * 8 * nd,
                            cudaMemcpyHostToDevice, s));
    g.discs_f = reinterpret_cast<const float4*>(ctx->discs_f.p);
    double lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1}, rmax = 0;
    for (int64_t i = 0; i < nd; ++i) {
      const double R = hd[7 * i + 6] * smax;
      rmax = std::max(rmax, R);
      for (int k = 0; k < 3; ++k) {
        lo[k] = std::min(lo[k], hd[7 * i + k] - R);
        hi[k] = std::max(hi[k], hd[7 * i + k] + R);
      }
    }
    double ext = std::max(hi[0] - lo[0], std::max(hi[1] - lo[1], hi[2] - lo[2]));
    // cells of twice the largest reach (half: 22 % slower on the cracked
    // cubes, a tet's box then spans more cells and meets discs again)
    double cell = std::max(2.0 * rmax, ext / 128.0);
    for (int k = 0; k < 3; ++k) {
      g.lo[k] = lo[k];
      g.dim[k] = std::max(1, (int)std::ceil((hi[k] - lo[k]) / cell));
    }
    g.inv_cell = 1.0 / cell;
    const int64_t cells = (int64_t)g.dim[0] * g.dim[1] * g.dim[2];
    DEC_TRY(ctx->grid_start.ensure(2 * (cells + 1)));
    int32_t* counts = ctx->grid_start.p;             // [cells+1] -> starts
    int32_t* cursor = ctx->grid_start.p + cells + 1;  // fill cursors
    DEC_TRY(cudaMemsetAsync(counts, 0, sizeof(int32_t) * (cells + 1), s));
    disc_bin_kernel<<<(unsigned)((nd + 127) / 128), 128, 0, s>>>(
        ctx->discs.p, (int)nd, smax, g, counts, cursor, nullptr, 0);
    DEC_TRY(cudaGetLastError());
    DEC_TRY(ctx->scan_tmp.ensure(scan_tmp_size(cells + 1)));
    DEC_TRY(exclusive_scan_u32((const uint32_t*)counts, (uint32_t*)counts, cells + 1,
                               ctx->scan_tmp.p, ctx->scan_tmp.cap, s));
    int32_t total = 0;
    DEC_TRY(cudaMemcpyAsync(&total, counts + cells, sizeof(int32_t),
                            cudaMemcpyDeviceToHost, s));
    DEC_TRY(cudaStreamSynchronize(s));
    DEC_TRY(ctx->grid_items.ensure(total > 0 ? total : 1));
    copy_i32_kernel<<<(unsigned)std::min<int64_t>((cells + 256) / 256, 4096), 256, 0, s>>>(
        counts, cursor, cells + 1);
    disc_bin_kernel<<<(unsigned)((nd + 127) / 128), 128, 0, s>>>(
        ctx->discs.p, (int)nd, smax, g, counts, cursor, ctx->grid_items.p, 1);
    DEC_TRY(cudaGetLastError());
    g.start = counts;
    g.items = ctx->grid_items.p;
    ctx->launches += 6;  // count, scan (3), cursor copy, fill
  }
  int64_t blocks = (m + 127) / 128;
  if (blocks > (int64_t)ctx->num_sms * 64) blocks = (int64_t)ctx->num_sms * 64;
  DEC_TRY(ctx->geom_count.ensure(1));
  DEC_TRY(cudaMemsetAsync(ctx->geom_count.p, 0, sizeof(unsigned long long), s));
  auto* kern = ctx->geom_precision == DEC_GEOM_MIXED ? hodge_tet_kernel<true>
                                                     : hodge_tet_kernel<false>;
  kern<<<(unsigned)std::max<int64_t>(blocks, 1), 128, 0, s>>>(
      ctx->xyz.p, ctx->tets.p, has_k ? ctx->kcond.p : nullptr,
      m, ctx->piece.p, has_k ? ctx->piece.p + q : nullptr, ctx->slot_cut.p, g,
      ctx->geom_count.p);
  DEC_TRY(cudaGetLastError());
  unsigned long long n64 = 0;
  DEC_TRY(cudaMemcpyAsync(&n64, ctx->geom_count.p, sizeof(n64), cudaMemcpyDeviceToHost, s));
  DEC_TRY(cudaStreamSynchronize(s));
  ctx->geom_fp64_tets = (int64_t)n64;
  int64_t eb = (ctx->ne + 255) / 256;
  if (eb > (int64_t)ctx->num_sms * 32) eb = (int64_t)ctx->num_sms * 32;
  edge_reduce_kernel<<<(unsigned)std::max<int64_t>(eb, 1), 256, 0, s>>>(
      ctx->seg_start.p, ctx->seg_pay.p, ctx->piece.p, has_k ? ctx->piece.p + q : nullptr, q,
      ctx->slot_cut.p, ctx->ne,
      ctx->w.p, ctx->first_cut.p);
  DEC_TRY(cudaGetLastError());
  ctx->launches += 2;
  if (n_fields > 1) {
    edge_reduce_fields_kernel<<<(unsigned)std::max<int64_t>(eb, 1), 256, 0, s>>>(
        ctx->seg_start.p, ctx->seg_pay.p, ctx->piece.p, ctx->piece.p + 2 * q, ctx->kcond.p, m,
        n_fields, ctx->ne, ctx->w.p);
    DEC_TRY(cudaGetLastError());
    ctx->launches += 1;
  }
  return DEC_OK;
}

}  // namespace dec
