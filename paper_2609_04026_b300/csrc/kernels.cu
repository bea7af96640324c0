// CUDA kernels of one LM step of holistic BA (sm_103a).
//
//   k_derive        per-entity data of a parameter set (rotation matrices, tangent bases)
//   k_linearize     K1: every residual of a feature and its IRLS weight; per-feature
//                   reduction of V_f = sum J_f^T w J_f, g_f, and per (feature, entity)
//                   slot W^T, the direct J_a^T w J_a block, J_a^T w r and, for cameras
//                   of a plane feature, J_cam^T w J_plane (thread per feature)
//   k_invert        K2: (V_f + lambda D_f) = L L^T by FP64 Cholesky; V^-1, L^-1, u_f = L^-1 g_f
//   k_whiten        K2: per slot Z = L^-1 W (double-single products) and b-part -G_e + Z^T u_f
//   k_schur_items   K3: atomic-free Schur accumulation.  Every upper block of S owns a
//                   list of slot pairs; each work item (<= 64 pairs) sums
//                   direct terms - Z_a^T Z_b in a fixed order into a partial
//   k_schur_blocks  K3: sums the partials of each block in order, adds lambda D on the
//                   diagonal, writes both triangles of the full block-CSR S and b
//   k_precond       K4: block-Jacobi inverse of the diagonal blocks of S (FP64 Cholesky)
//   k_pcg_*         K5/K6: PCG with a warp-per-block-row SpMV, FP64 vectors and dots, and
//                   a device-side stop flag so the host never waits inside the loop
//   k_backsub_slots K7: per slot W delta_a and its shares of g.delta, delta^T H delta
//   k_backsub       K7: delta_f = -V^-1 (g_f + sum W^T delta_a) and the predicted decrease
//                   -g.delta - 1/2 delta^T H delta from the stored blocks
//   k_candidate     K8: x (+) delta with the manifold retractions
//   k_cost          K8: FP64 robust cost of every residual, E and E_px
//   k_decide        K9: gain ratio, accept / reject, damping update
// All reductions are deterministic: warp shuffles in a fixed tree, per-block
// partials, and a last-arriving block that sums the partials in index order.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <math.h>

#include <mutex>
#include <type_traits>

#include "ba_internal.cuh"

namespace ba {

// ============================================================================
// deterministic reductions
// ============================================================================
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Reduce NV values over the grid.  Returns true in the last block to arrive (all
// of whose threads then hold the totals in `tot`).  `red` holds gridDim.x * NV doubles.
template <int NV>
__device__ bool grid_reduce(double (&v)[NV], double* red, unsigned int* counter, double (&tot)[NV]) {
  __shared__ double sh[32][NV];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = warp_sum(v[i]);
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) sh[wid][i] = v[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    double s[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) s[i] = 0;
    for (int w = 0; w < nw; ++w)
#pragma unroll
      for (int i = 0; i < NV; ++i) s[i] += sh[w][i];
#pragma unroll
    for (int i = 0; i < NV; ++i) red[(size_t)blockIdx.x * NV + i] = s[i];
    __threadfence();
    unsigned int t = atomicAdd(counter, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double s[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) s[i] = 0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
#pragma unroll
    for (int i = 0; i < NV; ++i) s[i] += __ldcg(&red[(size_t)b * NV + i]);
#pragma unroll
  for (int i = 0; i < NV; ++i) s[i] = warp_sum(s[i]);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) sh[wid][i] = s[i];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double a = 0;
    for (int w = 0; w < nw; ++w) a += sh[w][i];
    tot[i] = a;
  }
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

// ============================================================================
// small dense helpers
// ============================================================================
__host__ __device__ constexpr int up_idx(int i, int j, int k) { return i * k - i * (i - 1) / 2 + (j - i); }

// Cholesky inverse of an n x n SPD matrix given by its upper triangle (up_idx layout): A = L L^T,
// Linv = L^-1 (lower triangular) and Ainv = L^-T L^-1.  Returns false if a pivot is not positive.
template <int N>
__device__ bool chol_inverse(const double* Aup, double (&Ainv)[N][N], double (&Li)[N][N]) {
  double L[N][N];
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) L[i][j] = 0;
#pragma unroll
  for (int j = 0; j < N; ++j) {
    double s = Aup[up_idx(j, j, N)];
#pragma unroll
    for (int k = 0; k < j; ++k) s -= L[j][k] * L[j][k];
    if (!(s > 0)) return false;
    double ljj = sqrt(s);
    L[j][j] = ljj;
    double il = 1.0 / ljj;
#pragma unroll
    for (int i = j + 1; i < N; ++i) {
      double t = Aup[up_idx(j, i, N)];
#pragma unroll
      for (int k = 0; k < j; ++k) t -= L[i][k] * L[j][k];
      L[i][j] = t * il;
    }
  }
  // invert L (lower triangular)
#pragma unroll
  for (int i = 0; i < N; ++i) {
#pragma unroll
    for (int j = 0; j < N; ++j) Li[i][j] = 0;
    Li[i][i] = 1.0 / L[i][i];
#pragma unroll
    for (int j = 0; j < i; ++j) {
      double s = 0;
#pragma unroll
      for (int k = j; k < i; ++k) s += L[i][k] * Li[k][j];
      Li[i][j] = -s * Li[i][i];
    }
  }
  // A^-1 = L^-T L^-1
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = i; j < N; ++j) {
      double s = 0;
#pragma unroll
      for (int k = j; k < N; ++k) s += Li[k][i] * Li[k][j];
      Ainv[i][j] = s;
      Ainv[j][i] = s;
    }
  return true;
}

template <int N>
__device__ bool chol_inverse(const double* Aup, double (&Ainv)[N][N]) {
  double Li[N][N];
  return chol_inverse<N>(Aup, Ainv, Li);
}

// ============================================================================
// derived per-entity data
// ============================================================================
__device__ void quat_to_R(const double* q, double* R) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  double n = 1.0 / sqrt(w * w + x * x + y * y + z * z);
  w *= n; x *= n; y *= n; z *= n;
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z); R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z); R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y); R[7] = 2 * (y * z + w * x); R[8] = 1 - 2 * (x * x + y * y);
}

__device__ void tangent_basis_d(const double* n, double* b1, double* b2) {
  tangent_b1<double>(n, b1);
  cross3(n, b1, b2);
}

// cams: src n x 12 -> D (double) and optionally W (working type) with CAM_STRIDE
template <class T>
__device__ void derive_cam(const double* __restrict__ src, double* __restrict__ D, T* __restrict__ W, int64_t i) {
  const double* c = src + 12 * i;
  double o[17];
  quat_to_R(c, o);
  o[9] = c[4]; o[10] = c[5]; o[11] = c[6];
  o[12] = c[7]; o[13] = c[8]; o[14] = c[9]; o[15] = c[10]; o[16] = c[11];
  if (D)
    for (int k = 0; k < 17; ++k) D[CAM_STRIDE * i + k] = o[k];
  if (W)
    for (int k = 0; k < 17; ++k) W[CAM_STRIDE * i + k] = (T)o[k];
}

template <class T>
__global__ void k_derive_cams(int64_t nc, const double* __restrict__ src, double* __restrict__ D, T* __restrict__ W) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < nc) derive_cam<T>(src, D, W, i);
}

// groups: planes (n, w) then VPs v -> [n|v (3), w|0, b1 (3), b2 (3)] with GRP_STRIDE
template <class T>
__device__ void derive_group(int64_t npl, const double* __restrict__ pln, const double* __restrict__ vps,
                             double* __restrict__ D, T* __restrict__ W, int64_t i) {
  double o[10];
  if (i < npl) {
    const double* q = pln + 4 * i;
    o[0] = q[0]; o[1] = q[1]; o[2] = q[2]; o[3] = q[3];
  } else {
    const double* v = vps + 3 * (i - npl);
    o[0] = v[0]; o[1] = v[1]; o[2] = v[2]; o[3] = 0;
  }
  tangent_basis_d(o, o + 4, o + 7);
  if (D)
    for (int k = 0; k < 10; ++k) D[GRP_STRIDE * i + k] = o[k];
  if (W)
    for (int k = 0; k < 10; ++k) W[GRP_STRIDE * i + k] = (T)o[k];
}

template <class T>
__global__ void k_derive_groups(int64_t npl, int64_t nv, const double* __restrict__ pln, const double* __restrict__ vps,
                                double* __restrict__ D, T* __restrict__ W) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < npl + nv) derive_group<T>(npl, pln, vps, D, W, i);
}

__global__ void k_convert(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

cudaError_t launch_convert(cudaStream_t st, int64_t n, const double* a, float* b) {
  if (n <= 0) return cudaSuccess;
  k_convert<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, a, b);
  return cudaGetLastError();
}

// ============================================================================
// K1: linearise and reduce per feature
// ============================================================================
struct LossW {
  double w[N_KINDS];
  double a2[N_KINDS];
  double inv_a2[N_KINDS];   // 1 / a^2: the scaled squared norm s / a^2 as a product
  double half_wa2[N_KINDS]; // w a^2 / 2, the factor of the Cauchy cost
  float wf[N_KINDS], inv_a2f[N_KINDS];   // the float path's copies (no FP64 conversion per residual)
};
// the IRLS weight w / (1 + s / a^2) of a residual in the working type
template <class T>
__device__ __forceinline__ T irls_weight(const LossW& L, int kind, T s) {
  if constexpr (sizeof(T) == 4) return L.wf[kind] / (1.0f + s * L.inv_a2f[kind]);
  else return L.w[kind] / (1.0 + s * L.inv_a2[kind]);
}

template <class T>
struct LinArgs {
  const int8_t* rkind;
  const uint8_t* cam_mask;   // held pose components per camera (bit k = increment k)
  const int32_t *rcam, *rgrp, *rslot_c, *rslot_g, *fres_off, *feat_plane_slot;
  const int32_t *rslot_k, *fslot_off;   // refined intrinsics: per residual its intrinsics slot; slots per feature
  const uint8_t* slot_type;
  T* CK;                                // per camera slot J_cam^T w J_K of its own intrinsics entity
  const T* srf;                         // surface groups (SRF_STRIDE values each; sphere, cylinder, cone)
  T* CS;                                // per camera slot J_cam^T w J_group of the feature's surface group (SCS)
  int64_t nsp, ncy;                     // spheres, cylinders (the surface ids of cones follow)
  const T* bx;                          // ellipsoids then cuboids (BOX_STRIDE values each)
  int64_t nel;                          // ellipsoids
  const T* meas;
  const T *cam, *pts, *lin, *grp;
  int64_t npl, np;
  const int32_t* jp_pt;                 // 3D wireframe distance: per coupled point its point id
  int64_t nf;                           // points and lines (the coupled points' features follow)
  T *W, *H, *G, *C;
  double *V, *g;
  LossW loss;
};

// N values to a 16-byte aligned destination with 16-byte stores (a thread writes a whole record: one
// store instruction of a warp then carries 16 bytes per lane instead of 4)
template <class T, int N>
__device__ __forceinline__ void store16(T* __restrict__ dst, const T* src) {
  constexpr int V = 16 / (int)sizeof(T);
  constexpr int NV = N / V * V;
#pragma unroll
  for (int i = 0; i < NV; i += V) {
    if constexpr (sizeof(T) == 4)
      *reinterpret_cast<float4*>(dst + i) = make_float4(src[i], src[i + 1], src[i + 2], src[i + 3]);
    else
      *reinterpret_cast<double2*>(dst + i) = make_double2(src[i], src[i + 1]);
  }
  if constexpr (sizeof(T) == 4 && N - NV >= 2)
    *reinterpret_cast<float2*>(dst + NV) = make_float2(src[NV], src[NV + 1]);
  constexpr int NT2 = (sizeof(T) == 4 && N - NV >= 2) ? NV + 2 : NV;
#pragma unroll
  for (int i = NT2; i < N; ++i) dst[i] = src[i];
}

// N values from a 16-byte aligned record with 16-byte loads
template <class T, int N>
__device__ __forceinline__ void load16(const T* __restrict__ src, T* dst) {
  constexpr int V = 16 / (int)sizeof(T);
  constexpr int NV = N / V * V;
#pragma unroll
  for (int i = 0; i < NV; i += V) {
    if constexpr (sizeof(T) == 4) {
      const float4 t = *reinterpret_cast<const float4*>(src + i);
      dst[i] = t.x; dst[i + 1] = t.y; dst[i + 2] = t.z; dst[i + 3] = t.w;
    } else {
      const double2 t = *reinterpret_cast<const double2*>(src + i);
      dst[i] = t.x; dst[i + 1] = t.y;
    }
  }
  if constexpr (sizeof(T) == 4 && N - NV >= 2) {
    const float2 t = *reinterpret_cast<const float2*>(src + NV);
    dst[NV] = t.x; dst[NV + 1] = t.y;
  }
  constexpr int NT2 = (sizeof(T) == 4 && N - NV >= 2) ? NV + 2 : NV;
#pragma unroll
  for (int i = NT2; i < N; ++i) dst[i] = src[i];
}

// INTR: refined intrinsics (the residuals' intrinsics Jacobians, the intrinsics slots, the camera slots' couplings
// with their entities); WF: lines with 3D wireframe distances (their points' slots); SURF: the point kinds of
// spheres ... cuboids
template <class T, int KF, bool INTR = false, bool SURF = false, bool WF = false>
__device__ void linearize_feature(const LinArgs<T>& a, int64_t f) {
  constexpr bool XK = INTR || WF;   // the 3-dimension extra slots (intrinsics entities or coupled points)
  const int r0 = a.fres_off[f], r1 = a.fres_off[f + 1];
  // width of the positional group's accumulators: 3 (plane), 6 when spheres, cylinders or cones may occur
  constexpr int GW = SURF ? 6 : 3;
  constexpr int GH = GW * (GW + 1) / 2;
  constexpr int NV = KF * (KF + 1) / 2;
  T V[NV], gf[KF];
#pragma unroll
  for (int i = 0; i < NV; ++i) V[i] = 0;
#pragma unroll
  for (int i = 0; i < KF; ++i) gf[i] = 0;
  // current camera slot accumulators
  T Wc[KF][6], Hc[21], Gc[6], Cc[6][GW];
  int cur = -1;
  // group slot accumulators: the positional group (a plane, or a sphere / cylinder / cone: up to 6 dof), VP (2
  // dof, lines only)
  T Wp[KF][GW], Hp[GH], Gp[GW];
  T Wv[KF][2], Hv[3], Gv[2];
  int ps = -1, vs = -1;
#pragma unroll
  for (int i = 0; i < KF; ++i) {
#pragma unroll
    for (int j = 0; j < GW; ++j) Wp[i][j] = 0;
    Wv[i][0] = 0; Wv[i][1] = 0;
  }
#pragma unroll
  for (int i = 0; i < GH; ++i) Hp[i] = 0;
#pragma unroll
  for (int i = 0; i < GW; ++i) Gp[i] = 0;
  Hv[0] = Hv[1] = Hv[2] = 0;
  Gv[0] = Gv[1] = 0;
  const int plane_slot = a.feat_plane_slot[f];
  // the positional group is a sphere, cylinder, cone or a 9-parameter group (its camera couplings go to the
  // 6 x 6 CS records); a 9-parameter group's second entity has the next slot
  const bool surf = SURF && plane_slot >= 0 && ent_surface(a.slot_type[plane_slot]);
  const bool split = SURF && surf && plane_slot + 1 < a.fslot_off[f + 1] && ent_second(a.slot_type[plane_slot + 1]);
  // the second entity's accumulators (W, H, G), its coupling with the first (J_1^T w J_2) and with the current
  // camera (J_cam^T w J_2)
  T W2[KF][3], H2[6], G2[3], X12[6][3], C2[6][3];
  if constexpr (SURF) {
#pragma unroll
    for (int i = 0; i < KF; ++i) W2[i][0] = W2[i][1] = W2[i][2] = 0;
#pragma unroll
    for (int i = 0; i < 6; ++i) { H2[i] = 0; X12[i][0] = X12[i][1] = X12[i][2] = 0; C2[i][0] = C2[i][1] = C2[i][2] = 0; }
    G2[0] = G2[1] = G2[2] = 0;
  }

  T F[6];
  if (KF == 3) {
    const T* X = a.pts + 3 * f;
    F[0] = X[0]; F[1] = X[1]; F[2] = X[2];
  } else {
    const T* L = a.lin + 6 * (f - a.np);
#pragma unroll
    for (int i = 0; i < 6; ++i) F[i] = L[i];
  }

  auto flush = [&](int e) {
    store16<T, KF * 6>(a.W + (size_t)e * SW, &Wc[0][0]);
    T gh[SG];   // G (6), H (21), pad
#pragma unroll
    for (int i = 0; i < SG; ++i) gh[i] = i < HG_H ? Gc[i] : i < HG_H + 21 ? Hc[i - HG_H] : T(0);
    store16<T, SG>(a.G + (size_t)e * SG, gh);
    if constexpr (SURF) {
      if (surf) {
        T cb[SCS];
#pragma unroll
        for (int i = 0; i < SCS; ++i) cb[i] = Cc[i / 6][i % 6];
        store16<T, SCS>(a.CS + (size_t)e * SCS, cb);
      }
      if (split) {
        T cb[SC];
#pragma unroll
        for (int i = 0; i < SC; ++i) cb[i] = i < 18 ? C2[i / 3][i % 3] : T(0);
        store16<T, SC>(a.CK + (size_t)e * SC, cb);
#pragma unroll
        for (int i = 0; i < 6; ++i) C2[i][0] = C2[i][1] = C2[i][2] = 0;
      }
    }
    if (!surf && plane_slot >= 0) {
      T cb[SC];
#pragma unroll
      for (int i = 0; i < SC; ++i) cb[i] = i < 18 ? Cc[i / 3][i % 3] : T(0);
      store16<T, SC>(a.C + (size_t)e * SC, cb);
    }
  };
  auto zero_cam = [&]() {
#pragma unroll
    for (int i = 0; i < KF; ++i)
#pragma unroll
      for (int j = 0; j < 6; ++j) Wc[i][j] = 0;
#pragma unroll
    for (int i = 0; i < 21; ++i) Hc[i] = 0;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      Gc[i] = 0;
#pragma unroll
      for (int j = 0; j < GW; ++j) Cc[i][j] = 0;
    }
  };
  zero_cam();

  // refined intrinsics: the accumulators of the current intrinsics slot (W, G, the direct 3 x 3 block and the
  // coupling with the feature's plane), added into the slot's records whenever the slot changes (a slot may
  // recur: the residuals are in camera order and cameras may share an entity), and the current camera slot's
  // coupling with its own entity
  T Wk[KF][3], Gk[3], Hk[6], KPk[3][3], CKc[6][3];
  int curk = -1;
  auto zero_k = [&]() {
#pragma unroll
    for (int i = 0; i < KF; ++i) Wk[i][0] = Wk[i][1] = Wk[i][2] = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i) { Gk[i] = 0; KPk[i][0] = KPk[i][1] = KPk[i][2] = 0; }
#pragma unroll
    for (int i = 0; i < 6; ++i) Hk[i] = 0;
  };
  auto zero_ck = [&]() {
#pragma unroll
    for (int i = 0; i < 6; ++i) CKc[i][0] = CKc[i][1] = CKc[i][2] = 0;
  };
  auto add_k = [&](int e) {
    T wb[KF * 6], gh[SG], cb[SC];
    load16<T, KF * 6>(a.W + (size_t)e * SW, wb);
    load16<T, SG>(a.G + (size_t)e * SG, gh);
    load16<T, SC>(a.C + (size_t)e * SC, cb);
#pragma unroll
    for (int i = 0; i < KF; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) wb[i * 6 + j] += Wk[i][j];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      gh[i] += Gk[i];
#pragma unroll
      for (int j = i; j < 3; ++j) gh[HG_H + up_idx(i, j, 6)] += Hk[up_idx(i, j, 3)];
#pragma unroll
      for (int j = 0; j < 3; ++j) cb[i * 3 + j] += KPk[i][j];
    }
    store16<T, KF * 6>(a.W + (size_t)e * SW, wb);
    store16<T, SG>(a.G + (size_t)e * SG, gh);
    store16<T, SC>(a.C + (size_t)e * SC, cb);
  };
  if constexpr (XK) {
    zero_k();
    zero_ck();
    // the feature's extra slots start from zero (they are summed into below)
    const T z[SG > SC ? SG : SC] = {};
    for (int e = a.fslot_off[f]; e < a.fslot_off[f + 1]; ++e)
      if (a.slot_type[e] == ENT_INTR || a.slot_type[e] == ENT_JPT) {
        store16<T, KF * 6>(a.W + (size_t)e * SW, z);
        store16<T, SG>(a.G + (size_t)e * SG, z);
        store16<T, SC>(a.C + (size_t)e * SC, z);
      }
  }

  for (int rr = r0; rr < r1; ++rr) {
    const int kind = a.rkind[rr];
    const int sc = a.rslot_c[rr];
    if (sc != cur) {
      if constexpr (INTR) {
        if (cur >= 0) {
          T cb[SC];
#pragma unroll
          for (int i = 0; i < SC; ++i) cb[i] = i < 18 ? CKc[i / 3][i % 3] : T(0);
          store16<T, SC>(a.CK + (size_t)cur * SC, cb);
        }
        zero_ck();
      }
      if (cur >= 0) flush(cur);
      zero_cam();
      cur = sc;
    }
    if constexpr (XK) {
      const int sk = a.rslot_k[rr];
      if (sk != curk) {
        if (curk >= 0) add_k(curk);
        zero_k();
        curk = sk;
      }
    }
    const int camid = a.rcam[rr];
    const int gid = a.rgrp[rr];
    T meas[4];
    load16<T, 4>(a.meas + 4 * (size_t)rr, meas);
    Cam<T> c;
    if (camid >= 0) load_cam(a.cam + (size_t)CAM_STRIDE * camid, c);
    ResJ<T> o;
    if constexpr (SURF) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int k = 0; k < 6; ++k) o.Jg[i][k] = 0;   // a plane residual fills 3 of the 6 group columns
    }
    int rd = res_dim(kind);
    bool has_plane = false, has_vp = false;
    if (KF == 3) {
      if (kind == R_POINT) res_point<T, true, INTR>(c, F, meas, o);
      else if (kind == R_PLANE_POINT) { res_plane_point<T, true, INTR>(c, F, a.grp + (size_t)GRP_STRIDE * gid, o); has_plane = true; }
      else if (kind == R_P2L) res_p2l<T, true, INTR>(c, F, meas, o);
      else if (kind == R_PLANE_POINT3) { res_plane_point3<T, true>(F, a.grp + (size_t)GRP_STRIDE * gid, o); has_plane = true; }
      else if (SURF && kind == R_SPHERE_POINT) { res_surface_point<T, true, 0>(c, F, a.srf + (size_t)SRF_STRIDE * gid, o); has_plane = true; }
      else if (SURF && kind == R_CYL_POINT) { res_surface_point<T, true, 1>(c, F, a.srf + (size_t)SRF_STRIDE * (a.nsp + gid), o); has_plane = true; }
      else if (SURF && kind == R_CONE_POINT) { res_surface_point<T, true, 2>(c, F, a.srf + (size_t)SRF_STRIDE * (a.nsp + a.ncy + gid), o); has_plane = true; }
      else if (SURF && kind == R_ELL_POINT) { res_box_point<T, true, 3>(c, F, a.bx + (size_t)BOX_STRIDE * gid, o); has_plane = true; }
      else if (SURF && kind == R_CUB_POINT) { res_box_point<T, true, 4>(c, F, a.bx + (size_t)BOX_STRIDE * (a.nel + gid), o); has_plane = true; }
      else continue;
    } else {
      if (kind == R_LINE) res_line<T, true, INTR>(c, F, meas, o);
      else if (kind == R_PLANE_LINE) { res_plane_line<T, true, INTR>(c, F, a.grp + (size_t)GRP_STRIDE * gid, meas, o); has_plane = true; }
      else if (kind == R_VP) { res_vp<T, true, INTR>(F, a.grp + (size_t)GRP_STRIDE * (a.npl + gid), o); has_vp = true; }
      else if (kind == R_L2P) res_l2p<T, true, INTR>(c, F, meas, o);
      else if (kind == R_PLANE_LINE3) { res_plane_line3<T, true>(F, a.grp + (size_t)GRP_STRIDE * gid, o); has_plane = true; }
      else if (WF && kind == R_WF3D) res_wf3d<T, true>(F, a.pts + 3 * (size_t)gid, o);
      else if (SURF && kind == R_CUB_LINE) {
        res_box_line<T, true>(c, F, a.bx + (size_t)BOX_STRIDE * (a.nel + gid), meas, o);
        has_plane = true;
      }
      else continue;
    }
    if (!o.valid) continue;
    if (camid >= 0) {
      const unsigned held = a.cam_mask[camid];
      if (held)
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int k = 0; k < 6; ++k)
            if ((held >> k) & 1u) o.Jc[i][k] = 0;
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (i < rd) s += o.r[i] * o.r[i];
    const T om = irls_weight<T>(a.loss, kind, s);
    if (has_plane) ps = a.rslot_g[rr];
    if (has_vp) vs = a.rslot_g[rr];
    const bool camslot = sc >= 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (i >= rd) break;
      T wf[KF], wc[6], wg[GW];
#pragma unroll
      for (int k = 0; k < KF; ++k) wf[k] = om * o.Jf[i][k];
#pragma unroll
      for (int k = 0; k < 6; ++k) wc[k] = om * o.Jc[i][k];
#pragma unroll
      for (int k = 0; k < GW; ++k) wg[k] = om * o.Jg[i][k];
      const T ri = o.r[i];
      // V_f and g_f
#pragma unroll
      for (int p = 0; p < KF; ++p) {
        gf[p] += wf[p] * ri;
#pragma unroll
        for (int q = p; q < KF; ++q) V[up_idx(p, q, KF)] += wf[p] * o.Jf[i][q];
      }
      if (camslot) {
#pragma unroll
        for (int p = 0; p < KF; ++p)
#pragma unroll
          for (int q = 0; q < 6; ++q) Wc[p][q] += wf[p] * o.Jc[i][q];
#pragma unroll
        for (int p = 0; p < 6; ++p) {
          Gc[p] += wc[p] * ri;
#pragma unroll
          for (int q = p; q < 6; ++q) Hc[up_idx(p, q, 6)] += wc[p] * o.Jc[i][q];
        }
        if (has_plane)
#pragma unroll
          for (int p = 0; p < 6; ++p)
#pragma unroll
            for (int q = 0; q < GW; ++q) Cc[p][q] += wc[p] * o.Jg[i][q];
      }
      if (has_plane) {
#pragma unroll
        for (int p = 0; p < KF; ++p)
#pragma unroll
          for (int q = 0; q < GW; ++q) Wp[p][q] += wf[p] * o.Jg[i][q];
#pragma unroll
        for (int p = 0; p < GW; ++p) {
          Gp[p] += wg[p] * ri;
#pragma unroll
          for (int q = p; q < GW; ++q) Hp[up_idx(p, q, GW)] += wg[p] * o.Jg[i][q];
        }
      }
      if constexpr (SURF) {
        if (has_plane && (kind == R_ELL_POINT || kind == R_CUB_POINT || kind == R_CUB_LINE)) {
          // the 9-parameter group's second entity
          T w2[3];
#pragma unroll
          for (int k = 0; k < 3; ++k) w2[k] = om * o.Jg2[i][k];
#pragma unroll
          for (int p = 0; p < KF; ++p)
#pragma unroll
            for (int q = 0; q < 3; ++q) W2[p][q] += wf[p] * o.Jg2[i][q];
#pragma unroll
          for (int p = 0; p < 3; ++p) {
            G2[p] += w2[p] * ri;
#pragma unroll
            for (int q = p; q < 3; ++q) H2[up_idx(p, q, 3)] += w2[p] * o.Jg2[i][q];
          }
#pragma unroll
          for (int p = 0; p < 6; ++p)
#pragma unroll
            for (int q = 0; q < 3; ++q) X12[p][q] += wg[p] * o.Jg2[i][q];
          if (camslot)
#pragma unroll
            for (int p = 0; p < 6; ++p)
#pragma unroll
              for (int q = 0; q < 3; ++q) C2[p][q] += wc[p] * o.Jg2[i][q];
        }
      }
      if (KF == 4 && has_vp) {
#pragma unroll
        for (int p = 0; p < KF; ++p)
#pragma unroll
          for (int q = 0; q < 2; ++q) Wv[p][q] += wf[p] * o.Jg[i][q];
#pragma unroll
        for (int p = 0; p < 2; ++p) {
          Gv[p] += wg[p] * ri;
#pragma unroll
          for (int q = p; q < 2; ++q) Hv[up_idx(p, q, 2)] += wg[p] * o.Jg[i][q];
        }
      }
      if constexpr (XK) {
        if (curk >= 0) {
          T wk[3];
#pragma unroll
          for (int k = 0; k < 3; ++k) wk[k] = om * o.Jk[i][k];
#pragma unroll
          for (int p = 0; p < KF; ++p)
#pragma unroll
            for (int q = 0; q < 3; ++q) Wk[p][q] += wf[p] * o.Jk[i][q];
#pragma unroll
          for (int p = 0; p < 3; ++p) {
            Gk[p] += wk[p] * ri;
#pragma unroll
            for (int q = p; q < 3; ++q) Hk[up_idx(p, q, 3)] += wk[p] * o.Jk[i][q];
          }
          if (has_plane)
#pragma unroll
            for (int p = 0; p < 3; ++p)
#pragma unroll
              for (int q = 0; q < 3; ++q) KPk[p][q] += wk[p] * o.Jg[i][q];
          if (camslot)
#pragma unroll
            for (int p = 0; p < 6; ++p)
#pragma unroll
              for (int q = 0; q < 3; ++q) CKc[p][q] += wc[p] * o.Jk[i][q];
        }
      }
    }
  }
  if constexpr (XK) {
    if (cur >= 0) {
      T cb[SC];
#pragma unroll
      for (int i = 0; i < SC; ++i) cb[i] = i < 18 ? CKc[i / 3][i % 3] : T(0);
      store16<T, SC>(a.CK + (size_t)cur * SC, cb);
    }
    if (curk >= 0) add_k(curk);
  }
  if (cur >= 0) flush(cur);
  // group slots, padded to the 6-wide block of the reduced system
  // W (stride ws per feature row) and the upper H (dimension hd) of a group slot; nd real dimensions
  auto put_group = [&](int e, int nd, const T* Wg, int ws, const T* Hg, int hd, const T* Gg) {
    T wb[KF * 6], gh[SG];   // W; G (6), H (21), pad
#pragma unroll
    for (int i = 0; i < KF; ++i)
#pragma unroll
      for (int j = 0; j < 6; ++j) wb[i * 6 + j] = j < nd ? Wg[i * ws + j] : T(0);
#pragma unroll
    for (int i = 0; i < SG; ++i) gh[i] = T(0);
#pragma unroll
    for (int i = 0; i < 6; ++i) gh[i] = i < nd ? Gg[i] : T(0);
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int j = i; j < 6; ++j)
        if (j < nd) gh[HG_H + up_idx(i, j, 6)] = Hg[up_idx(i, j, hd)];
    store16<T, KF * 6>(a.W + (size_t)e * SW, wb);
    store16<T, SG>(a.G + (size_t)e * SG, gh);
  };
  if (ps < 0) ps = plane_slot;  // a plane slot whose residuals were all invalid
  if (ps >= 0) put_group(ps, SURF ? ent_dims(a.slot_type[ps]) : 3, &Wp[0][0], GW, Hp, GW, Gp);
  if constexpr (SURF) {
    if (split) {
      put_group(plane_slot + 1, 3, &W2[0][0], 3, H2, 3, G2);
      T cb[SC];
#pragma unroll
      for (int i = 0; i < SC; ++i) cb[i] = i < 18 ? X12[i / 3][i % 3] : T(0);
      store16<T, SC>(a.C + (size_t)(plane_slot + 1) * SC, cb);
    }
  }
  if (KF == 4) {
    if (vs < 0) {
      // find the VP slot (if any) among this feature's residuals
      for (int rr = r0; rr < r1; ++rr)
        if (a.rkind[rr] == R_VP) { vs = a.rslot_g[rr]; break; }
    }
    if (vs >= 0) put_group(vs, 2, &Wv[0][0], 2, Hv, 2, Gv);
  }
  double vb[NV], gbf[KF];
#pragma unroll
  for (int i = 0; i < NV; ++i) vb[i] = (double)V[i];
#pragma unroll
  for (int i = 0; i < KF; ++i) gbf[i] = (double)gf[i];
  store16<double, NV>(a.V + 10 * f, vb);
  store16<double, KF>(a.g + 4 * f, gbf);
}

template <class T, int KF, bool INTR = false, bool SURF = false, bool WF = false>
__global__ void __launch_bounds__(128) k_linearize(LinArgs<T> a, int64_t f0, int64_t f1) {
  int64_t f = f0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f < f1) linearize_feature<T, KF, INTR, SURF, WF>(a, f);
}

// The residuals of a point that the 3D wireframe distance makes an entity of A (a zero-dimension feature: no
// W, V or g): per camera slot its G, H, the coupling with the point (CK record) and with the plane (C record);
// the point slot's G, H and its coupling with the plane (C record, J_point^T w J_plane, 3 x 3); the plane
// slot's G, H.  Point kinds with a camera or the direct plane distance (the other group types are refused
// together with this distance).
template <class T>
__device__ void linearize_jpoint(const LinArgs<T>& a, int64_t q) {
  const int64_t f = a.nf + q;
  const int r0 = a.fres_off[f], r1 = a.fres_off[f + 1];
  const T* X = a.pts + 3 * (size_t)a.jp_pt[q];
  const T F[3] = {X[0], X[1], X[2]};
  T Hc[21], Gc[6], Cc[6][3], CKc[6][3];
  T Hk[6], Gk[3], KP[3][3], Hp[6], Gp[3];
  int cur = -1, ps = -1, sk = -1;
  auto zero_cam = [&]() {
#pragma unroll
    for (int i = 0; i < 21; ++i) Hc[i] = 0;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      Gc[i] = 0;
#pragma unroll
      for (int j = 0; j < 3; ++j) { Cc[i][j] = 0; CKc[i][j] = 0; }
    }
  };
  auto flush = [&](int e) {
    T gh[SG];
#pragma unroll
    for (int i = 0; i < SG; ++i) gh[i] = i < HG_H ? Gc[i] : i < HG_H + 21 ? Hc[i - HG_H] : T(0);
    store16<T, SG>(a.G + (size_t)e * SG, gh);
    T cb[SC];
#pragma unroll
    for (int i = 0; i < SC; ++i) cb[i] = i < 18 ? Cc[i / 3][i % 3] : T(0);
    store16<T, SC>(a.C + (size_t)e * SC, cb);
#pragma unroll
    for (int i = 0; i < SC; ++i) cb[i] = i < 18 ? CKc[i / 3][i % 3] : T(0);
    store16<T, SC>(a.CK + (size_t)e * SC, cb);
  };
  zero_cam();
#pragma unroll
  for (int i = 0; i < 6; ++i) { Hk[i] = 0; Hp[i] = 0; }
#pragma unroll
  for (int i = 0; i < 3; ++i) { Gk[i] = 0; Gp[i] = 0; KP[i][0] = KP[i][1] = KP[i][2] = 0; }
  for (int rr = r0; rr < r1; ++rr) {
    const int kind = a.rkind[rr];
    const int sc = a.rslot_c[rr];
    if (sc != cur) {
      if (cur >= 0) flush(cur);
      zero_cam();
      cur = sc;
    }
    sk = a.rslot_k[rr];
    const int camid = a.rcam[rr];
    const int gid = a.rgrp[rr];
    T meas[4];
    load16<T, 4>(a.meas + 4 * (size_t)rr, meas);
    Cam<T> c;
    if (camid >= 0) load_cam(a.cam + (size_t)CAM_STRIDE * camid, c);
    ResJ<T> o;
    bool has_plane = false;
    if (kind == R_POINT) res_point<T, true>(c, F, meas, o);
    else if (kind == R_PLANE_POINT) { res_plane_point<T, true>(c, F, a.grp + (size_t)GRP_STRIDE * gid, o); has_plane = true; }
    else if (kind == R_P2L) res_p2l<T, true>(c, F, meas, o);
    else if (kind == R_PLANE_POINT3) { res_plane_point3<T, true>(F, a.grp + (size_t)GRP_STRIDE * gid, o); has_plane = true; }
    else continue;
    if (!o.valid) continue;
    if (camid >= 0) {
      const unsigned held = a.cam_mask[camid];
      if (held)
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int k = 0; k < 6; ++k)
            if ((held >> k) & 1u) o.Jc[i][k] = 0;
    }
    const int rd = res_dim(kind);
    T s = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (i < rd) s += o.r[i] * o.r[i];
    const T om = irls_weight<T>(a.loss, kind, s);
    if (has_plane) ps = a.rslot_g[rr];
    const bool camslot = sc >= 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (i >= rd) break;
      T wx[3], wc[6], wg[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) { wx[k] = om * o.Jf[i][k]; wg[k] = om * o.Jg[i][k]; }
#pragma unroll
      for (int k = 0; k < 6; ++k) wc[k] = om * o.Jc[i][k];
      const T ri = o.r[i];
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        Gk[p] += wx[p] * ri;
#pragma unroll
        for (int q2 = p; q2 < 3; ++q2) Hk[up_idx(p, q2, 3)] += wx[p] * o.Jf[i][q2];
      }
      if (camslot) {
#pragma unroll
        for (int p = 0; p < 6; ++p) {
          Gc[p] += wc[p] * ri;
#pragma unroll
          for (int q2 = p; q2 < 6; ++q2) Hc[up_idx(p, q2, 6)] += wc[p] * o.Jc[i][q2];
#pragma unroll
          for (int q2 = 0; q2 < 3; ++q2) CKc[p][q2] += wc[p] * o.Jf[i][q2];
        }
        if (has_plane)
#pragma unroll
          for (int p = 0; p < 6; ++p)
#pragma unroll
            for (int q2 = 0; q2 < 3; ++q2) Cc[p][q2] += wc[p] * o.Jg[i][q2];
      }
      if (has_plane) {
#pragma unroll
        for (int p = 0; p < 3; ++p) {
          Gp[p] += wg[p] * ri;
#pragma unroll
          for (int q2 = p; q2 < 3; ++q2) Hp[up_idx(p, q2, 3)] += wg[p] * o.Jg[i][q2];
#pragma unroll
          for (int q2 = 0; q2 < 3; ++q2) KP[p][q2] += wx[p] * o.Jg[i][q2];
        }
      }
    }
  }
  if (cur >= 0) flush(cur);
  // the point slot (the feature's last) and the plane slot: G and the upper H in the 6-wide layout
  auto put3 = [&](int e, const T* Gg, const T* Hg) {
    T gh[SG];
#pragma unroll
    for (int i = 0; i < SG; ++i) gh[i] = T(0);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      gh[i] = Gg[i];
#pragma unroll
      for (int j = i; j < 3; ++j) gh[HG_H + up_idx(i, j, 6)] = Hg[up_idx(i, j, 3)];
    }
    store16<T, SG>(a.G + (size_t)e * SG, gh);
  };
  if (sk < 0 && r1 > r0) sk = a.fslot_off[f + 1] - 1;
  if (sk >= 0) {
    put3(sk, Gk, Hk);
    T cb[SC];
#pragma unroll
    for (int i = 0; i < SC; ++i) cb[i] = i < 9 ? KP[i / 3][i % 3] : T(0);
    store16<T, SC>(a.C + (size_t)sk * SC, cb);
  }
  if (ps < 0) ps = a.feat_plane_slot[f];
  if (ps >= 0) put3(ps, Gp, Hp);
}

template <class T>
__global__ void __launch_bounds__(128) k_linearize_jpoint(LinArgs<T> a, int64_t njp) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q < njp) linearize_jpoint<T>(a, q);
}

// ============================================================================
// K2: damped landmark inverse, the whitened slot blocks Z = L^-1 W and the per-slot b parts
// ============================================================================
template <class T>
struct InvArgs {
  const int32_t *fslot_off, *slot_feat;
  const double *V, *g;
  const T *W, *G;
  double *Vinv, *u, *L;
  T *Z, *B;
  int64_t np, nf, ne;
  double lambda;
  DevScalars* S;
};

template <int K>
__device__ void invert_damped(const double* Vup, double lambda, double (&Vi)[K][K], double (&Li)[K][K], int* flag) {
  double A[K * (K + 1) / 2];
#pragma unroll
  for (int i = 0; i < K * (K + 1) / 2; ++i) A[i] = Vup[i];
#pragma unroll
  for (int i = 0; i < K; ++i) {
    double dgi = fmin(fmax(A[up_idx(i, i, K)], 1e-6), 1e32);
    A[up_idx(i, i, K)] += lambda * dgi;
  }
  if (!chol_inverse<K>(A, Vi, Li)) {
    // rounding made the damped block indefinite: add damping until it factorises
    *flag = 1;
    double tr = 0;
#pragma unroll
    for (int i = 0; i < K; ++i) tr += fabs(A[up_idx(i, i, K)]);
    double extra = 1e-12 * tr + 1e-300;
    for (int t = 0; t < 60; ++t) {
#pragma unroll
      for (int i = 0; i < K; ++i) A[up_idx(i, i, K)] += extra;
      if (chol_inverse<K>(A, Vi, Li)) return;
      extra *= 10;
    }
#pragma unroll
    for (int i = 0; i < K; ++i)
#pragma unroll
      for (int j = 0; j < K; ++j) { Vi[i][j] = 0; Li[i][j] = 0; }
  }
}

// Z = L^-1 W for one slot (K x 6, rows of W at stride 6).  With a float working type the product is
// formed in double-single arithmetic on the float pipes (L^-1 split into hi + lo floats, exact products
// by FMA, TwoSum accumulation) and rounded to float once: rounding V^-1 or L^-1 to float before the
// product would multiply the error by the condition number of V_f, and the Schur complement of a
// poorly observed feature then loses the cancellation that makes its contribution small.
template <int K>
__device__ __forceinline__ void whiten_slot(const double (&Li)[K][K], const double* W, double* Z) {
#pragma unroll
  for (int i = 0; i < K; ++i)
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      double s = 0;
#pragma unroll
      for (int k = 0; k <= i; ++k) s = fma(Li[i][k], W[k * 6 + j], s);
      Z[i * 6 + j] = s;
    }
}
template <int K>
__device__ __forceinline__ void whiten_slot(const float (&Lh)[K][K], const float (&Ll)[K][K], const float* W, float* Z) {
#pragma unroll
  for (int i = 0; i < K; ++i)
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      float hi = 0, lo = 0;
#pragma unroll
      for (int k = 0; k <= i; ++k) {
        const float w = W[k * 6 + j];
        const float ph = Lh[i][k] * w;
        const float pe = fmaf(Lh[i][k], w, -ph);
        const float sm = hi + ph;
        const float bp = sm - hi;
        lo += ((hi - (sm - bp)) + (ph - bp)) + fmaf(Ll[i][k], w, pe);
        hi = sm;
      }
      Z[i * 6 + j] = hi + lo;
    }
}

// the damped landmark inverse of one feature: V^-1 (for the back-substitution), L^-1 and u = L^-1 g_f
template <class T, int K>
__device__ void invert_core(const InvArgs<T>& a, int64_t f, double (&Li)[K][K], T (&ut)[K]) {
  double Vi[K][K];
  int flag = 0;
  invert_damped<K>(a.V + 10 * f, a.lambda, Vi, Li, &flag);
  if (flag) atomicOr(&a.S->flags, 1);
  double* vo = a.Vinv + 10 * f;
#pragma unroll
  for (int i = 0; i < K; ++i)
#pragma unroll
    for (int j = i; j < K; ++j) vo[up_idx(i, j, K)] = Vi[i][j];
  // u = L^-1 g_f: the slot's share of b is -G_e + Z_e^T u  (= -G_e + W_e^T V^-1 g_f)
#pragma unroll
  for (int i = 0; i < K; ++i) {
    double s = 0;
#pragma unroll
    for (int k = 0; k <= i; ++k) s += Li[i][k] * a.g[4 * f + k];
    a.u[4 * f + i] = s;
    ut[i] = (T)s;
  }
}

template <class T, int K>
__device__ __forceinline__ void split_L(const double (&Li)[K][K], T (&Lh)[K][K], T (&Ll)[K][K]) {
#pragma unroll
  for (int i = 0; i < K; ++i)
#pragma unroll
    for (int j = 0; j < K; ++j) {
      Lh[i][j] = (T)Li[i][j];
      Ll[i][j] = (T)(Li[i][j] - (double)Lh[i][j]);
    }
}

// one slot: Z_e = L^-1 W_e and the slot's share of b
template <class T, int K>
__device__ __forceinline__ void whiten_record(const InvArgs<T>& a, int64_t e, const double (&Li)[K][K], const T (&Lh)[K][K],
                                              const T (&Ll)[K][K], const T (&ut)[K]) {
  T w[K * 6], z[K * 6], G[6];
  load16<T, K * 6>(a.W + (size_t)e * SW, w);
  if constexpr (sizeof(T) == 8) whiten_slot<K>(Li, (const double*)w, (double*)z);
  else whiten_slot<K>(Lh, Ll, w, z);
  store16<T, K * 6>(a.Z + (size_t)e * SW, z);
  load16<T, 6>(a.G + (size_t)e * SG, G);
  T* B = a.B + (size_t)e * SB;
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    T s = -G[j];
#pragma unroll
    for (int k = 0; k < K; ++k) s += z[k * 6 + j] * ut[k];
    B[j] = s;
  }
}

// a whole feature in one thread (the batched-window kernel)
template <class T, int K>
__device__ void invert_feature(const InvArgs<T>& a, int64_t f) {
  double Li[K][K];
  T ut[K], Lh[K][K], Ll[K][K];
  invert_core<T, K>(a, f, Li, ut);
  split_L<T, K>(Li, Lh, Ll);
  for (int e = a.fslot_off[f]; e < a.fslot_off[f + 1]; ++e) whiten_record<T, K>(a, e, Li, Lh, Ll, ut);
}

// grid path: a thread per feature factors the block and stores L^-1 (lower triangle, up_idx of the
// transpose), then a thread per slot whitens that slot, so that slot records stream coalesced
template <class T, int K>
__device__ void invert_store(const InvArgs<T>& a, int64_t f) {
  double Li[K][K];
  T ut[K];
  invert_core<T, K>(a, f, Li, ut);
  double* lo = a.L + 10 * f;
#pragma unroll
  for (int i = 0; i < K; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) lo[up_idx(j, i, K)] = Li[i][j];
}

template <class T>
__global__ void __launch_bounds__(128) k_invert(InvArgs<T> a) {
  int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= a.nf) return;
  if (f < a.np) invert_store<T, 3>(a, f);
  else invert_store<T, 4>(a, f);
}

template <class T, int K>
__device__ __forceinline__ void whiten_from_store(const InvArgs<T>& a, int64_t e, int64_t f) {
  double Li[K][K];
  T ut[K], Lh[K][K], Ll[K][K];
  const double* lo = a.L + 10 * f;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    ut[i] = (T)a.u[4 * f + i];
#pragma unroll
    for (int j = 0; j < K; ++j) Li[i][j] = j <= i ? lo[up_idx(j, i, K)] : 0.0;
  }
  split_L<T, K>(Li, Lh, Ll);
  whiten_record<T, K>(a, e, Li, Lh, Ll, ut);
}

template <class T>
__global__ void __launch_bounds__(128) k_whiten(InvArgs<T> a) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= a.ne) return;
  const int64_t f = a.slot_feat[e];
  if (f >= a.nf) {
    // a slot of a wireframe-coupled point's residuals (a zero-dimension feature): Z = 0, the b part -G
    const T z[SW] = {};
    store16<T, SW>(a.Z + (size_t)e * SW, z);
    T G[6];
    load16<T, 6>(a.G + (size_t)e * SG, G);
#pragma unroll
    for (int j = 0; j < 6; ++j) a.B[(size_t)e * SB + j] = -G[j];
  } else if (f < a.np) {
    whiten_from_store<T, 3>(a, e, f);
  } else {
    whiten_from_store<T, 4>(a, e, f);
  }
}

// ============================================================================
// K3: Schur complement, atomic-free
// ============================================================================
// Every upper block of S owns the list of slot pairs (e_a, e_b) of the features that see both of its
// entities, in feature order; the list is cut into work units of at most UNIT_MAX pairs.  A unit sums
//   sum over its pairs of  direct(e_a, e_b) - Z_a^T Z_b        (W_a V^-1 W_b^T = (L^-1 W_a)^T (L^-1 W_b))
// entry by entry in pair order, where direct() is the slot's J_a^T w J_a block on the diagonal and the
// camera-plane block J_cam^T w J_plane of a plane feature (pair_b bit 31).  A float working type sums in
// double-single arithmetic across lanes.  An off-diagonal block that fits one unit is written to S with
// its mirror directly; the units of a diagonal block or of a longer block leave FP64 partials that a
// finishing pass adds in unit order before the damping.  The grid path and the batched-window path run
// the same warp-level unit code, so both form every entry with the same operations in the same order.
template <class T>
struct BlockArgs {
  const int32_t *up_row, *up_full, *up_mirror, *col;
  const uint8_t *ent_type, *cam_fixed;
  T* Sval;
  SView sv;        // where each block of S is stored (full or typed storage)
  double *b, *Dg, *sdiag;
  const double *relH, *relG;   // inter-group relations: per group entity J^T w J (36) and J^T w r (6), or null
  int64_t nc, ngend;           // cameras; end of the group entities (planes and VPs; intrinsics entities follow)
  double lambda;
};

template <class T>
struct UnitArgs {
  const int32_t *un_se, *un_blk, *un_order, *up_un, *pair_a, *pair_b, *multi;
  const int4* un_desc;      // per unit in processing order: first pair, end pair, block position, unit id
  const int32_t* un_mflag;  // per unit in processing order: mirror position << 2 | written directly << 1 | diagonal
  const int4* pk_desc;      // per pack of small units: first unit (processing order), units, first pair, pairs
  const T *Z, *H, *B, *C;
  const T* CK;     // refined intrinsics: per camera slot J_cam^T w J_K of its own entity (or null)
  const T* CS;     // surface groups: per camera slot J_cam^T w J_group of the feature's sphere / cylinder / cone
  double* upart;   // 48 per unit: 36 S, 6 b, 6 diag(H)
  int* ctr;        // grid path: the next unit a warp takes (zero at launch)
  int64_t nun, nmulti, nun_main, npack;
  int line_slot0;
  BlockArgs<T> fb;
};

// running sum of a unit's terms: FP64 for a double working type; for float a double-single (hi, lo)
// pair with TwoSum, since a warp-wide FP64 add or conversion costs dozens of float instructions on
// this part.  value() rounds once to double, rounded() once to float.
template <class T>
struct PartSum;
template <>
struct PartSum<double> {
  double s = 0;
  __device__ __forceinline__ void add(double v) { s += v; }
  __device__ __forceinline__ double value() const { return s; }
  __device__ __forceinline__ double rounded() const { return s; }
};
template <>
struct PartSum<float> {
  float hi = 0, lo = 0;
  __device__ __forceinline__ void add(float v) {
    const float sm = hi + v;
    const float bp = sm - hi;
    lo += (hi - (sm - bp)) + (v - bp);
    hi = sm;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
  __device__ __forceinline__ float rounded() const { return hi + lo; }
};


// acc - (Z_a^T Z_b)_ij (rows at stride 6), the products fused into the running sum (three FMAs for a point's records, four for a
// line's), so that every kernel forms it identically
template <class T>
__device__ __forceinline__ T pair_sub(T acc, const T* za, const T* zb, int i, int j, bool line) {
  acc = fma(-za[i], zb[j], acc);
  acc = fma(-za[6 + i], zb[6 + j], acc);
  acc = fma(-za[12 + i], zb[12 + j], acc);
  if (line) acc = fma(-za[18 + i], zb[18 + j], acc);
  return acc;
}


// direct term of entry (i, j) for a pair of a diagonal block or a camera-plane pair
template <class T>
__device__ __forceinline__ T pair_direct(const UnitArgs<T>& a, int ea, bool diag, bool cam_plane, int i, int j) {
  if (diag) return a.H[(size_t)ea * SH + (i <= j ? up_idx(i, j, 6) : up_idx(j, i, 6))];
  if (cam_plane && j < 3) return a.C[(size_t)ea * SC + i * 3 + j];
  return T(0);
}

// a diagonal block of S from its sums: symmetric part, damping lambda D on the real dimensions, a unit
// diagonal on padding and held camera components; writes S, b, D and the diagonal of S
template <class T>
__device__ void finish_diag(const BlockArgs<T>& a, int row, int fpos, double (&s)[36], double (&bb)[6],
                            double (&hh)[6]) {
  // a group's inter-group relations (direct terms of H_gg and g_g, Section 3.2), before the damping
  if (a.relH && row >= a.nc && row < a.ngend) {
    const double* H = a.relH + 36 * (size_t)(row - a.nc);
    const double* G = a.relG + 6 * (size_t)(row - a.nc);
#pragma unroll
    for (int e = 0; e < 36; ++e) s[e] += H[e];
#pragma unroll
    for (int i = 0; i < 6; ++i) { bb[i] -= G[i]; hh[i] += H[7 * i]; }
  }
  // Z_e^T Z_e is symmetric by construction and so is H_e; the symmetric part is taken anyway so
  // that CG always sees an exactly symmetric S
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = i + 1; j < 6; ++j) {
      const double m = 0.5 * (s[i * 6 + j] + s[j * 6 + i]);
      s[i * 6 + j] = m;
      s[j * 6 + i] = m;
    }
  const int nd = ent_dims(a.ent_type[row]);
  const unsigned held = (row < a.nc) ? a.cam_fixed[row] : 0u;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    bool real = i < nd && !((held >> i) & 1u);
    double Di = real ? fmin(fmax(hh[i], 1e-6), 1e32) : 1.0;
    a.Dg[6 * (size_t)row + i] = Di;
    if (real) {
      s[i * 6 + i] += a.lambda * Di;
      a.b[6 * (size_t)row + i] = bb[i];
    } else {
      // padding (or a held camera): unit diagonal, no coupling, zero right-hand side
#pragma unroll
      for (int j = 0; j < 6; ++j) { s[i * 6 + j] = 0; s[j * 6 + i] = 0; }
      s[i * 6 + i] = 1;
      a.b[6 * (size_t)row + i] = 0;
    }
  }
  const BlkTarget tg = sview_target(a.sv, fpos);   // a diagonal block is stored whole (6 x 6)
#pragma unroll
  for (int i = 0; i < 36; ++i) a.Sval[tg.off + i] = (T)s[i];
#pragma unroll
  for (int i = 0; i < 6; ++i) a.sdiag[6 * (size_t)row + i] = (double)(T)s[i * 6 + i];
}

// a diagonal block, or a block split over several units: FP64 sum of the unit partials in unit order
template <class T>
__device__ void unit_finish(const UnitArgs<T>& a, int u) {
  const int row = a.fb.up_row[u], fpos = a.fb.up_full[u];
  const bool diag = a.fb.col[fpos] == row;
  double s[36], bb[6], hh[6];
#pragma unroll
  for (int i = 0; i < 36; ++i) s[i] = 0;
#pragma unroll
  for (int i = 0; i < 6; ++i) { bb[i] = 0; hh[i] = 0; }
  for (int w = a.up_un[u]; w < a.up_un[u + 1]; ++w) {
    const double* p = a.upart + (size_t)w * 48;
#pragma unroll
    for (int i = 0; i < 36; ++i) s[i] += p[i];
    if (diag)
#pragma unroll
      for (int i = 0; i < 6; ++i) { bb[i] += p[36 + i]; hh[i] += p[42 + i]; }
  }
  if (diag) {
    finish_diag<T>(a.fb, row, fpos, s, bb, hh);
    return;
  }
  const int mpos = a.fb.up_mirror[u];
  const BlkTarget tm = sview_target(a.fb.sv, fpos), tt = sview_target(a.fb.sv, mpos);
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const T v = (T)s[i * 6 + j];
      if (j < tm.w) a.fb.Sval[tm.off + i * tm.w + j] = v;
      if (i < tt.w) a.fb.Sval[tt.off + j * tt.w + i] = v;
    }
}

template <class T>
__global__ void __launch_bounds__(128) k_schur_finish(UnitArgs<T> a) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k < a.nmulti) unit_finish<T>(a, a.multi[k]);
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// A warp per work unit; lane l takes pairs l, l + 32, ... of the unit.  For each stage of 32 pairs the
// warp gathers both Z records of every pair into shared memory with 16-byte cp.async copies (each lane
// keeps up to a dozen copies in flight); every lane then adds the full 6 x 6 term of its pair to its own
// accumulators in the working type.  At the end the lanes' accumulators are summed across lanes in lane
// order (double-single for float), and lane l writes entry l (and 32 + l) of the block.
// Shared memory per warp: 32 staged pairs at a padded stride (conflict-free 16-byte loads) and the pair
// indices; the stage area is reused for the cross-lane sums.
template <class T>
struct UnitSmem {
  static constexpr int stride = sizeof(T) == 4 ? 52 : 50;   // elements per staged pair: Z_a | Z_b | pad
  static constexpr int red = 49;                            // row stride of the cross-lane sums (36 + 12 + 1)
  static constexpr size_t bytes = sizeof(T) * 32 * stride + 2 * 32 * sizeof(int);
};

template <class T>
__device__ __forceinline__ void load_rec(const T* src, T (&z)[24], bool line) {
  if constexpr (sizeof(T) == 4) {
    const float4* q = reinterpret_cast<const float4*>(src);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      if (k == 5 && !line) { z[20] = 0; z[21] = 0; z[22] = 0; z[23] = 0; continue; }   // a point has 3 rows
      const float4 t = q[k];
      z[4 * k] = t.x; z[4 * k + 1] = t.y; z[4 * k + 2] = t.z; z[4 * k + 3] = t.w;
    }
  } else {
    const double2* q = reinterpret_cast<const double2*>(src);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      if (k >= 9 && !line) { z[2 * k] = 0; z[2 * k + 1] = 0; continue; }
      const double2 t = q[k];
      z[2 * k] = t.x; z[2 * k + 1] = t.y;
    }
  }
}

// the running sums of one work unit in a lane: the 6 x 6 term (and, for a diagonal block, b and diag(H))
template <class T>
struct UnitAcc {
  T acc[36], bacc[6], hacc[6];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int e = 0; e < 36; ++e) acc[e] = 0;
#pragma unroll
    for (int i = 0; i < 6; ++i) { bacc[i] = 0; hacc[i] = 0; }
  }
};

// the pair indices of the stage [base, base + n) into sa_ / sb_ and the 16-byte copies of both Z records of
// every pair into the stage buffer (cp.async; the caller waits)
// A diagonal block's pairs are (e, e): their stage holds the Z record once and, after it, the slot's direct
// block H (for float the whole G|H record, whose start is 16-byte aligned; for double H and its pad, from
// offset HG_H); DiagStage gives the copy's source offset from H, its 16-byte pieces and where H lands
template <class T>
struct DiagStage {
  static constexpr int src = sizeof(T) == 4 ? -HG_H : 0;        // from a.H + e * SH
  static constexpr int pieces = sizeof(T) == 4 ? SG * 4 / 16 : 22 * 8 / 16;
  static constexpr int h_at = SW + (sizeof(T) == 4 ? HG_H : 0);  // H in the staged pair
  static_assert(SW + pieces * 16 / (int)sizeof(T) <= UnitSmem<T>::stride, "a diagonal pair fits its stage slot");
};

template <class T>
__device__ __forceinline__ void unit_stage_issue(const UnitArgs<T>& a, bool diag, int base, int n, T* stage, int* sa_,
                                                 int* sb_, int lane) {
  constexpr int ST = UnitSmem<T>::stride;
  constexpr int CH = SW * (int)sizeof(T) / 16;   // 16-byte pieces of one Z record
  constexpr int DP = DiagStage<T>::pieces;
  if (lane < n) { sa_[lane] = a.pair_a[base + lane]; sb_[lane] = a.pair_b[base + lane]; }
  __syncwarp();
  if (diag) {
    for (int t = lane; t < n * (CH + DP); t += 32) {
      const int p = t / (CH + DP), r = t - p * (CH + DP);
      const int e = sa_[p];
      if (r < CH)
        cp_async16(reinterpret_cast<char*>(stage + p * ST) + 16 * r,
                   reinterpret_cast<const char*>(a.Z + (size_t)e * SW) + 16 * r);
      else
        cp_async16(reinterpret_cast<char*>(stage + p * ST + SW) + 16 * (r - CH),
                   reinterpret_cast<const char*>(a.H + (size_t)e * SH + DiagStage<T>::src) + 16 * (r - CH));
    }
    return;
  }
  for (int t = lane; t < n * 2 * CH; t += 32) {
    const int p = t / (2 * CH), r = t - p * 2 * CH;
    const int which = r / CH, ch = r - which * CH;
    const int e = which == 0 ? sa_[p] : (sb_[p] & PAIR_SLOT);
    cp_async16(reinterpret_cast<char*>(stage + p * ST + which * SW) + 16 * ch,
               reinterpret_cast<const char*>(a.Z + (size_t)e * SW) + 16 * ch);
  }
}

// lane's term of its pair (lane < n) of a staged stage, added to its running sums
// a diagonal pair's b part (the slot's B record), loaded before the stage's copies are waited for
template <class T>
__device__ __forceinline__ void unit_diag_b(const UnitArgs<T>& a, bool diag, int n, const int* sa_, int lane, T (&bv)[6]) {
  if (diag && lane < n) {
    const T* Bv = a.B + (size_t)sa_[lane] * SB;
#pragma unroll
    for (int i = 0; i < 6; ++i) bv[i] = Bv[i];
  }
}

template <class T>
__device__ __forceinline__ void unit_stage_compute(const UnitArgs<T>& a, bool diag, int n, const T* stage,
                                                   const int* sa_, const int* sb_, int lane, const T (&bv)[6],
                                                   UnitAcc<T>& u) {
  constexpr int ST = UnitSmem<T>::stride;
  if (lane >= n) return;
  T* acc = u.acc;
  const int ea = sa_[lane];
  const unsigned code = (unsigned)sb_[lane] >> PAIR_SHIFT;
  const bool line = ea >= a.line_slot0;
  T za[24], zb[24];
  load_rec(stage + lane * ST, za, line);
  if (diag) {
    // the pair (e, e): one staged Z record, the staged H after it
#pragma unroll
    for (int k = 0; k < 24; ++k) zb[k] = za[k];
    const T* H = stage + lane * ST + DiagStage<T>::h_at;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      u.bacc[i] += bv[i];
      u.hacc[i] += H[up_idx(i, i, 6)];
#pragma unroll
      for (int j = 0; j < 6; ++j) acc[i * 6 + j] = pair_sub(acc[i * 6 + j] + H[i <= j ? up_idx(i, j, 6) : up_idx(j, i, 6)], za, zb, i, j, line);
    }
    return;
  }
  load_rec(stage + lane * ST + SW, zb, line);
  if (code == PAIR_CP || code == PAIR_CK) {
    // the camera's direct block with the plane, or with its own intrinsics entity (6 x 3)
    const T* Cm = (code == PAIR_CP ? a.C : a.CK) + (size_t)ea * SC;
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int j = 0; j < 6; ++j) acc[i * 6 + j] = pair_sub(acc[i * 6 + j] + (j < 3 ? Cm[i * 3 + j] : T(0)), za, zb, i, j, line);
  } else if (code == PAIR_CS) {
    // the camera's direct block with the feature's sphere, cylinder or cone (6 x 6, zeros beyond its dims)
    const T* Cm = a.CS + (size_t)ea * SCS;
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int j = 0; j < 6; ++j) acc[i * 6 + j] = pair_sub(acc[i * 6 + j] + Cm[i * 6 + j], za, zb, i, j, line);
  } else if (code == PAIR_G12) {
    // a 9-parameter group's two entities: the second entity's slot holds J_1^T w J_2 (6 x 3)
    const T* Cm = a.C + (size_t)(sb_[lane] & PAIR_SLOT) * SC;
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int j = 0; j < 6; ++j) acc[i * 6 + j] = pair_sub(acc[i * 6 + j] + (j < 3 ? Cm[i * 3 + j] : T(0)), za, zb, i, j, line);
  } else if (code == PAIR_PK) {
    // plane-intrinsics: the intrinsics slot holds J_K^T w J_plane (3 x 3); this block is its transpose
    const T* Cm = a.C + (size_t)(sb_[lane] & PAIR_SLOT) * SC;
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int j = 0; j < 6; ++j) acc[i * 6 + j] = pair_sub(acc[i * 6 + j] + (i < 3 && j < 3 ? Cm[j * 3 + i] : T(0)), za, zb, i, j, line);
  } else {
#pragma unroll
    for (int e = 0; e < 36; ++e) acc[e] = pair_sub(acc[e], za, zb, e / 6, e % 6, line);
  }
}

// the unit's cross-lane sums in lane order (red: 32 x RS values of shared memory, free to overwrite), written to
// S directly (a block this unit covers alone) or as FP64 partials of the unit
template <class T>
__device__ __forceinline__ void unit_finish_warp(const UnitArgs<T>& a, int fpos, int w, int mf, T* red, int lane,
                                                 const UnitAcc<T>& u) {
  constexpr int RS = UnitSmem<T>::red;
  const bool diag = (mf & 1) != 0;
  const bool direct = (mf & 2) != 0;
#pragma unroll
  for (int e = 0; e < 36; ++e) red[lane * RS + e] = u.acc[e];
  if (diag)
#pragma unroll
    for (int i = 0; i < 6; ++i) { red[lane * RS + 36 + i] = u.bacc[i]; red[lane * RS + 42 + i] = u.hacc[i]; }
  __syncwarp();
  const int ne = diag ? 48 : 36;
  const int mpos = mf >> 2;
  BlkTarget tm{0, 0}, tt{0, 0};
  if (direct) { tm = sview_target(a.fb.sv, fpos); tt = sview_target(a.fb.sv, mpos); }
  for (int e = lane; e < ne; e += 32) {
    PartSum<T> sm;
    for (int k = 0; k < 32; ++k) sm.add(red[k * RS + e]);
    if (!direct) {
      a.upart[(size_t)w * 48 + e] = sm.value();
    } else {
      const T v = (T)sm.rounded();
      const int i = e / 6, j = e % 6;
      if (j < tm.w) a.fb.Sval[tm.off + i * tm.w + j] = v;
      if (i < tt.w) a.fb.Sval[tt.off + j * tt.w + i] = v;
    }
  }
  __syncwarp();
}

template <class T>
__device__ void unit_warp(const UnitArgs<T>& a, int g, char* smem, int lane) {
  constexpr int ST = UnitSmem<T>::stride;
  T* stage = reinterpret_cast<T*>(smem);
  int* sa_ = reinterpret_cast<int*>(smem + sizeof(T) * 32 * ST);
  int* sb_ = sa_ + 32;
  // the unit's descriptor (two independent loads instead of a chain through the block's arrays)
  const int4 dsc = a.un_desc[g];
  const int mf = a.un_mflag[g];
  const int s0 = dsc.x, s1 = dsc.y, fpos = dsc.z, w = dsc.w;
  const bool diag = (mf & 1) != 0;
  UnitAcc<T> u;
  u.zero();
  for (int base = s0; base < s1; base += 32) {
    const int n = min(32, s1 - base);
    unit_stage_issue<T>(a, diag, base, n, stage, sa_, sb_, lane);
    T bv[6];
    unit_diag_b<T>(a, diag, n, sa_, lane, bv);
    cp_async_wait_all();
    __syncwarp();
    unit_stage_compute<T>(a, diag, n, stage, sa_, sb_, lane, bv, u);
    __syncwarp();   // the next stage overwrites the staged records
  }
  unit_finish_warp<T>(a, fpos, w, mf, stage, lane, u);   // the stage area takes the cross-lane sums
}

// Grid path: persistent warps, each taking the next unit of the processing order from a counter, with the
// stages of its units in a two-deep pipeline: the copies of the next stage (of this unit or of the next) are
// in flight while the current stage is summed, so a warp waits for a stage's gather only when the sums of
// the previous one took less time.  Every unit's sums are those of unit_warp.
template <class T>
struct UnitPipeSmem {
  static constexpr size_t buf = UnitSmem<T>::bytes;   // a stage buffer and its pair indices
  static constexpr size_t bytes = 2 * buf;
};

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

template <class T>
__device__ void unit_pipe_warp(const UnitArgs<T>& a, char* smem, int lane) {
  constexpr int ST = UnitSmem<T>::stride;
  constexpr size_t BUF = UnitPipeSmem<T>::buf;
  auto stage_of = [&](int b) { return reinterpret_cast<T*>(smem + b * BUF); };
  auto sa_of = [&](int b) { return reinterpret_cast<int*>(smem + b * BUF + sizeof(T) * 32 * ST); };
  auto take = [&]() {
    int v = 0;
    if (lane == 0) v = atomicAdd(a.ctr, 1);
    return __shfl_sync(0xffffffffu, v, 0);
  };
  int g = take();
  if (g >= a.nun_main) return;
  int4 dsc = a.un_desc[g];
  int mf = a.un_mflag[g];
  int base = dsc.x;
  int buf = 0;
  UnitAcc<T> u;
  u.zero();
  unit_stage_issue<T>(a, (mf & 1) != 0, base, min(32, dsc.y - base), stage_of(0), sa_of(0), sa_of(0) + 32, lane);
  cp_async_commit();
  for (;;) {
    // the next stage: the rest of this unit, else the first of the warp's next unit
    const bool last = base + 32 >= dsc.y;
    int ng = g, nbase = base + 32;
    int4 nd = dsc;
    int nmf = mf;
    if (last) {
      ng = take();
      if (ng < a.nun_main) { nd = a.un_desc[ng]; nmf = a.un_mflag[ng]; nbase = nd.x; }
    }
    const bool more = ng < a.nun_main;
    T bv[6];
    unit_diag_b<T>(a, (mf & 1) != 0, min(32, dsc.y - base), sa_of(buf), lane, bv);
    if (more) {
      __syncwarp();   // the other buffer's last readers are done
      unit_stage_issue<T>(a, (nmf & 1) != 0, nbase, min(32, nd.y - nbase), stage_of(buf ^ 1), sa_of(buf ^ 1),
                          sa_of(buf ^ 1) + 32, lane);
      cp_async_commit();
      cp_async_wait_prev();
    } else {
      cp_async_wait_all();
    }
    __syncwarp();
    const int* sa_ = sa_of(buf);
    unit_stage_compute<T>(a, (mf & 1) != 0, min(32, dsc.y - base), stage_of(buf), sa_, sa_ + 32, lane, bv, u);
    __syncwarp();
    if (last) {
      unit_finish_warp<T>(a, dsc.z, dsc.w, mf, stage_of(buf), lane, u);
      u.zero();
      if (!more) break;
      g = ng; dsc = nd; mf = nmf;
    }
    base = nbase;
    buf ^= 1;
  }
}

template <class T>
struct UnitWarps { static constexpr int n = sizeof(T) == 4 ? 4 : 2; };

// grid path: persistent warps over the units in the unit order (long units first), pipelined stages
template <class T>
__global__ void __launch_bounds__(UnitWarps<T>::n * 32) k_schur_units(UnitArgs<T> a) {
  constexpr int NW = UnitWarps<T>::n;
  extern __shared__ __align__(16) char unit_dyn[];   // NW x UnitPipeSmem<T>::bytes
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unit_pipe_warp<T>(a, unit_dyn + (size_t)warp * UnitPipeSmem<T>::bytes, lane);
}

// persistent grid of the unit kernel: the CTAs that are resident at once (opted in to its shared memory)
template <class T>
int schur_units_grid(int device, int64_t nun_main) {
  constexpr int NW = UnitWarps<T>::n;
  static int per_sm[2][64] = {};
  const int ti = sizeof(T) == 4 ? 0 : 1;
  if (device < 0 || device >= 64) device = 0;
  const size_t smem = (size_t)NW * UnitPipeSmem<T>::bytes;
  if (!per_sm[ti][device]) {
    cudaFuncSetAttribute(k_schur_units<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int nb = 0, sms = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_schur_units<T>, NW * 32, smem);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaGetLastError();
    per_sm[ti][device] = std::max(1, nb) * std::max(1, sms);
  }
  return (int)std::min<int64_t>(per_sm[ti][device], (nun_main + NW - 1) / NW);
}

// Small units, several to a warp: a pack holds whole off-diagonal blocks of a few pairs each (not
// camera-plane blocks), their pairs contiguous, one pair per lane.  Lane l forms the term of pair l, and
// each block's 36 entries are summed over its own lanes in lane order, then written to S with the mirror.
// A lane's term and the order of the sums are those of unit_warp for the same block (which adds only
// zeros beyond its pairs), so both paths give identical blocks; a warp no longer spends a stage and a
// 32-lane sum on a block of a handful of pairs.
template <class T>
struct PackSmem {
  static constexpr int stride = UnitSmem<T>::stride;
  // per warp, a multiple of 16 bytes so that every warp's stage is 16-byte aligned (cp.async, 16-byte loads)
  static constexpr size_t bytes = (sizeof(T) * 32 * stride + sizeof(int) * (33 + 32 + 32 + 32 + 32) + 15) / 16 * 16;
  static_assert(sizeof(T) * 32 * stride % 16 == 0, "stage area must keep 16-byte alignment");
};
static_assert(PackSmem<float>::bytes % 16 == 0 && PackSmem<double>::bytes % 16 == 0, "warp areas must be 16-byte aligned");
static_assert(UnitSmem<float>::bytes % 16 == 0 && UnitSmem<double>::bytes % 16 == 0, "warp areas must be 16-byte aligned");

template <class T>
__global__ void __launch_bounds__(UnitWarps<T>::n * 32) k_schur_packs(UnitArgs<T> a) {
  constexpr int NW = UnitWarps<T>::n;
  constexpr int ST = UnitSmem<T>::stride, RS = UnitSmem<T>::red;
  constexpr int CH = SW * (int)sizeof(T) / 16;
  __shared__ __align__(16) char smem[NW][PackSmem<T>::bytes];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t pk = blockIdx.x * (int64_t)NW + warp;
  if (pk >= a.npack) return;   // the whole warp leaves together
  T* stage = reinterpret_cast<T*>(smem[warp]);
  int* seg = reinterpret_cast<int*>(smem[warp] + sizeof(T) * 32 * ST);   // first lane of each block (+ end)
  int* fp = seg + 33;   // block position
  int* mp = fp + 32;    // mirror position
  int* sa_ = mp + 32;
  int* sb_ = sa_ + 32;
  const int4 pd = a.pk_desc[pk];
  const int nu = pd.y, p0 = pd.z, n = pd.w;
  if (lane < nu) {
    const int4 dd = a.un_desc[pd.x + lane];
    seg[lane] = dd.x - p0;
    fp[lane] = dd.z;
    mp[lane] = a.un_mflag[pd.x + lane] >> 2;
  }
  if (lane == 0) seg[nu] = n;
  if (lane < n) { sa_[lane] = a.pair_a[p0 + lane]; sb_[lane] = a.pair_b[p0 + lane]; }
  __syncwarp();
  for (int t = lane; t < n * 2 * CH; t += 32) {
    const int p = t / (2 * CH), r = t - p * 2 * CH;
    const int which = r / CH, ch = r - which * CH;
    const int e = which == 0 ? sa_[p] : (sb_[p] & PAIR_SLOT);   // packed pairs carry no direct-block code
    cp_async16(reinterpret_cast<char*>(stage + p * ST + which * SW) + 16 * ch,
               reinterpret_cast<const char*>(a.Z + (size_t)e * SW) + 16 * ch);
  }
  cp_async_wait_all();
  __syncwarp();
  T acc[36];
  if (lane < n) {
    const bool line = sa_[lane] >= a.line_slot0;
    T za[24], zb[24];
    load_rec(stage + lane * ST, za, line);
    load_rec(stage + lane * ST + SW, zb, line);
#pragma unroll
    for (int e = 0; e < 36; ++e) acc[e] = pair_sub(T(0), za, zb, e / 6, e % 6, line);
  }
  __syncwarp();   // the staged records are overwritten by the terms
  T* red = stage;
  if (lane < n)
#pragma unroll
    for (int e = 0; e < 36; ++e) red[lane * RS + e] = acc[e];
  __syncwarp();
  for (int t = lane; t < nu * 36; t += 32) {
    const int i = t / 36, e = t - 36 * i;
    PartSum<T> sm;
    for (int k = seg[i]; k < seg[i + 1]; ++k) sm.add(red[k * RS + e]);
    const T v = (T)sm.rounded();
    const BlkTarget tm = sview_target(a.fb.sv, fp[i]), tt = sview_target(a.fb.sv, mp[i]);
    const int ei = e / 6, ej = e % 6;
    if (ej < tm.w) a.fb.Sval[tm.off + ei * tm.w + ej] = v;
    if (ei < tt.w) a.fb.Sval[tt.off + ej * tt.w + ei] = v;
  }
}

// ============================================================================
// K4: block-Jacobi preconditioner
// ============================================================================
// SOA: S in the library's padded interleaved storage; otherwise 36 contiguous values per block
template <class T, bool SOA>
__device__ void precond_row(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                            const T* __restrict__ Sval, T* __restrict__ Minv, DevScalars* S, int64_t a,
                            const SView& sv) {
  int pos = -1;
  for (int q = row_ptr[a]; q < row_ptr[a + 1]; ++q)
    if (col[q] == a) { pos = q; break; }
  // the diagonal block is stored whole in either storage
  const int64_t dof = SOA ? sview_target(sv, pos).off : (int64_t)pos * BS2;
  double Aup[21];
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = i; j < 6; ++j) Aup[up_idx(i, j, 6)] = (double)Sval[dof + i * 6 + j];
  double Mi[6][6];
  if (!chol_inverse<6>(Aup, Mi)) {
    atomicOr(&S->flags, 4);
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int j = 0; j < 6; ++j) Mi[i][j] = (i == j && Aup[up_idx(i, i, 6)] > 0) ? 1.0 / Aup[up_idx(i, i, 6)] : (i == j ? 1.0 : 0.0);
  }
  T* o = Minv + (size_t)a * BS2;
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = 0; j < 6; ++j) o[i * 6 + j] = (T)Mi[i][j];
}

template <class T, bool SOA>
__global__ void k_precond(int64_t na, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                          const T* __restrict__ Sval, T* __restrict__ Minv, DevScalars* S, SView sv) {
  int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a < na) precond_row<T, SOA>(row_ptr, col, Sval, Minv, S, a, sv);
}

// ============================================================================
// K5/K6: preconditioned conjugate gradients
// ============================================================================
template <class T>
__device__ __forceinline__ void apply_block(const T* __restrict__ M, const double* __restrict__ v, double* o) {
  T vv[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) vv[j] = (T)v[j];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    T s = 0;
#pragma unroll
    for (int j = 0; j < 6; ++j) s += M[i * 6 + j] * vv[j];
    o[i] = (double)s;
  }
}

// Persistent PCG: one cooperative launch runs the whole solve.  Every CTA owns a
// contiguous range of block rows (balanced by stored blocks); rows are cut into
// chunks of <= PCG_CHUNK blocks that the CTA's warps multiply (FP32 / working-type
// products, FP64 sums of the block results), and a warp sums a row's chunk partials
// in order, so y = S p is deterministic.  Three grid-wide barriers per iteration:
// after the SpMV (alpha needs p.Ap), after the update (beta and the stop test need
// r.r and r.z), and after p = z + beta p (the next SpMV reads every p).  Every CTA
// forms the global sums from the same per-CTA partials in the same order, so all
// CTAs take the same stop decision.
// Accumulator of the SpMV products S_ij p_j.  With double S (FP64 path) it is a plain
// double.  With float S (mixed path) it is a double-single pair (hi, lo) of floats:
// p_j is split into hi + lo floats, S_ij * hi is formed exactly as a product and its
// FMA-recovered rounding error (TwoProduct, Dekker 1971), and the sum is kept with
// Knuth's TwoSum, so the float pipes deliver products accurate to ~1e-14 relative.
// Plain float products lose the strong cancellation of S p (a Laplacian-like operator
// whose row sums nearly vanish) and CG then stops converging.
template <class T>
struct DotAcc;

template <>
struct DotAcc<double> {
  double s = 0;
  __device__ __forceinline__ double value() const { return s; }
};

template <>
struct DotAcc<float> {
  float hi = 0, lo = 0;
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ void block_dot6(const double* __restrict__ B, const double* x, DotAcc<double> (&acc)[6]) {
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = 0; j < 6; ++j) acc[i].s = fma(B[i * 6 + j], x[j], acc[i].s);
}

// one block's 6 row products with the (head, tail) operand: each row's 6-term dot product in float FMA (its
// rounding is a few units of the block's own float entries, the order of their storage rounding), added to
// the double-single row sum once
__device__ __forceinline__ void block_dot6_split(const float* __restrict__ B, const float* xh, const float* xl,
                                                 DotAcc<float> (&acc)[6]) {
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    float h = 0.f, l = 0.f;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      h = fmaf(B[i * 6 + j], xh[j], h);
      l = fmaf(B[i * 6 + j], xl[j], l);
    }
    const float sm = acc[i].hi + h;   // TwoSum(hi, h), the tails added to the error
    const float bp = sm - acc[i].hi;
    const float er = (acc[i].hi - (sm - bp)) + (h - bp);
    acc[i].hi = sm;
    acc[i].lo = acc[i].lo + l + er;
  }
}

__device__ __forceinline__ void block_dot6(const float* __restrict__ B, const double* x, DotAcc<float> (&acc)[6]) {
  float xh[6], xl[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    xh[j] = (float)x[j];
    xl[j] = (float)(x[j] - (double)xh[j]);
  }
  block_dot6_split(B, xh, xl, acc);
}

// warp sum of a product accumulator, left in lane 0.  Double-single lanes are combined with TwoSum
// on the float pipes and stay double-single: on this part a warp-wide FP64 instruction costs as
// much as dozens of float ones, so conversions to double happen once per block row, not per chunk.
__device__ __forceinline__ DotAcc<double> warp_sum_acc(const DotAcc<double>& a) {
  DotAcc<double> r;
  r.s = warp_sum(a.s);
  return r;
}
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float h2, float l2) {
  const float sm = hi + h2;
  const float bp = sm - hi;
  const float er = (hi - (sm - bp)) + (h2 - bp);
  hi = sm;
  lo = lo + l2 + er;
}
__device__ __forceinline__ DotAcc<float> warp_sum_acc(const DotAcc<float>& a) {
  float hi = a.hi, lo = a.lo;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float h2 = __shfl_down_sync(0xffffffffu, hi, o);
    const float l2 = __shfl_down_sync(0xffffffffu, lo, o);
    two_sum_acc(hi, lo, h2, l2);
  }
  DotAcc<float> r;
  r.hi = hi;
  r.lo = lo;
  return r;
}
// running sum of chunk results in the accumulator's own precision
__device__ __forceinline__ void acc_add(DotAcc<double>& s, const DotAcc<double>& v) { s.s += v.s; }
__device__ __forceinline__ void acc_add(DotAcc<float>& s, const DotAcc<float>& v) { two_sum_acc(s.hi, s.lo, v.hi, v.lo); }

__device__ __forceinline__ float2 split2(double v) {
  const float h = (float)v;
  return make_float2(h, (float)(v - (double)h));
}

// the 36 values of one stored block (16-byte aligned: a block is 144 or 288 bytes)
__device__ __forceinline__ void load_block36(const float* p, float (&B)[36]) {
  const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const float4 t = q[k];
    B[4 * k] = t.x; B[4 * k + 1] = t.y; B[4 * k + 2] = t.z; B[4 * k + 3] = t.w;
  }
}
__device__ __forceinline__ void load_block36(const double* p, double (&B)[36]) {
  const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
  for (int k = 0; k < 18; ++k) {
    const double2 t = q[k];
    B[2 * k] = t.x; B[2 * k + 1] = t.y;
  }
}

template <class T>
struct PcgArgs;

template <class T>
struct PcgArgs {
  int64_t na;
  const int32_t *col, *cta_row0, *row_chunk0, *chunk_beg;
  const T *Sval, *Minv;
  const double* b;
  double *x, *r, *z, *p, *Ap;
  float2* phl;   // float working type: p split into (hi, lo) floats, written where p is written
  double* part;  // 3 x G x 2 per-CTA partial sums
  DevScalars* S;
  double tol;
  int max_iters;
  long long budget;   // clock64 cycles a grid barrier may wait
};

// one stored block times the gathered p block: FP64 FMAs for double S; for float S the pre-split
// (hi, lo) copy of p feeds the double-single products without any FP64 instruction
__device__ __forceinline__ void spmv_block(const double* B, const PcgArgs<double>& a, int col, DotAcc<double> (&acc)[6]) {
  const double* pb = a.p + 6 * (size_t)col;
  double xv[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) xv[j] = __ldcg(&pb[j]);
  block_dot6(B, xv, acc);
}

__device__ __forceinline__ void spmv_block(const float* B, const PcgArgs<float>& a, int col, DotAcc<float> (&acc)[6]) {
  const float2* pb = a.phl + 6 * (size_t)col;
  float xh[6], xl[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const float2 v = __ldcg(&pb[j]);
    xh[j] = v.x;
    xl[j] = v.y;
  }
  block_dot6_split(B, xh, xl, acc);
}

template <int NT>
__device__ __forceinline__ void cta_sum2(double v0, double v1, double* out2) {
  __shared__ double sh[NT / 32][2];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v0 = warp_sum(v0);
  v1 = warp_sum(v1);
  if (lane == 0) { sh[w][0] = v0; sh[w][1] = v1; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, c = 0;
    for (int i = 0; i < NT / 32; ++i) { a += sh[i][0]; c += sh[i][1]; }
    out2[0] = a; out2[1] = c;
  }
  __syncthreads();
}

// sum of the G per-CTA partials (2 values), identical in every CTA; result broadcast in bc
__device__ __forceinline__ void grid_partials2(const double* part, int G, double* bc) {
  if (threadIdx.x < 32) {
    double a = 0, c = 0;
    for (int g = threadIdx.x; g < G; g += 32) { a += __ldcg(&part[2 * g]); c += __ldcg(&part[2 * g + 1]); }
    a = warp_sum(a);
    c = warp_sum(c);
    if (threadIdx.x == 0) { bc[0] = a; bc[1] = c; }
  }
  __syncthreads();
}

// ---- a grid barrier for the persistent PCG kernels.  The launch is cooperative, so every CTA is resident;
// the wait is still bounded, by `budget` clock64 cycles (ba_options.wait_budget_cycles).  A CTA whose wait
// runs out records PCG_FLAG_TIMEOUT.  The result is the same for every thread of the CTA: false when this
// CTA's wait ran out or any CTA has recorded a timeout, and the kernel then leaves its iteration.  The
// arrival count is reset on the host before every launch; the generation word only ever advances.
__device__ __forceinline__ bool grid_barrier(DevScalars* S, unsigned G, long long budget) {
  __shared__ int ok_sh;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* genp = &S->bar_gen;
    const unsigned g0 = *genp;
    __threadfence();
    int ok = 1;
    if (atomicAdd(&S->bar_count, 1u) == G - 1) {
      atomicExch(&S->bar_count, 0u);
      __threadfence();
      atomicAdd(&S->bar_gen, 1u);
    } else {
      const long long t0 = clock64();
      while (*genp == g0)
        if (clock64() - t0 > budget) { ok = 0; break; }
    }
    __threadfence();
    if (!ok) atomicOr(&S->flags, PCG_FLAG_TIMEOUT);
    if (*(volatile int*)&S->flags & PCG_FLAG_TIMEOUT) ok = 0;
    ok_sh = ok;
  }
  __syncthreads();
  return ok_sh != 0;
}

// ---- the typed and stream PCGs' grid barrier: one arrival counter that only grows within a launch (reset on
// the host before it), so that the k-th barrier of a launch is passed once the counter reaches k x G.  The last arrival
// needs one atomic round trip and the waiters one load to see it (no reset of the count, no generation word).
// A CTA that must end the solve (a copy wait or this wait ran out) adds BAR_ABORT: every CTA then leaves at its
// current or next barrier with false, and PCG_FLAG_TIMEOUT is recorded for the host.
constexpr unsigned long long BAR_ABORT = 1ull << 40;
__device__ __forceinline__ bool grid_barrier_count(DevScalars* S, unsigned long long target, bool abort_cta,
                                                   long long budget) {
  __shared__ int ok_sh;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();   // the CTA's writes before its arrival
    const unsigned long long add = abort_cta ? BAR_ABORT + 1ull : 1ull;
    unsigned long long v = atomicAdd(&S->bar_arrive, add) + add;
    int ok = 1;
    if (v < target) {
      volatile unsigned long long* cp = &S->bar_arrive;
      const long long t0 = clock64();
      while ((v = *cp) < target)
        if (clock64() - t0 > budget) {
          ok = 0;
          atomicOr(&S->flags, PCG_FLAG_TIMEOUT);
          atomicAdd(&S->bar_arrive, BAR_ABORT);
          break;
        }
    }
    __threadfence();   // the other CTAs' writes before their arrivals
    if (v >= BAR_ABORT) ok = 0;
    ok_sh = ok;
  }
  __syncthreads();
  return ok_sh != 0;
}

// SOA: S in the padded interleaved storage, chunks of exactly 32 blocks (one per lane, coalesced
// loads); otherwise contiguous blocks and chunks of up to PCG_CHUNK blocks strided over the lanes
template <class T, int NT, bool SOA>
__global__ void __launch_bounds__(NT, 1) k_pcg_persistent(PcgArgs<T> a) {
  extern __shared__ double chunk_mem[];   // [chunks of this CTA][6] accumulators
  DotAcc<T>* chunk_y = reinterpret_cast<DotAcc<T>*>(chunk_mem);
  __shared__ double bc[2];
  __shared__ double cta_out[2];
  const int G = gridDim.x, c = blockIdx.x;
  const int r0 = a.cta_row0[c], r1 = a.cta_row0[c + 1];
  const int q0 = a.row_chunk0[r0], q1 = a.row_chunk0[r1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int NW = NT / 32;
  double* partA = a.part;
  double* partB = a.part + 2 * G;
  double* partC = a.part + 4 * G;

  // ---- init: x = 0, r = b, z = M^-1 r, p = z
  double v0 = 0, v1 = 0;
  for (int row = r0 + threadIdx.x; row < r1; row += NT) {
    double rv[6], zv[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) { rv[i] = a.b[6 * row + i]; a.x[6 * row + i] = 0; a.r[6 * row + i] = rv[i]; }
    apply_block(a.Minv + (size_t)row * BS2, rv, zv);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      a.z[6 * row + i] = zv[i];
      a.p[6 * row + i] = zv[i];
      if (a.phl) a.phl[6 * row + i] = split2(zv[i]);
      v0 += rv[i] * zv[i];
      v1 += rv[i] * rv[i];
    }
  }
  cta_sum2<NT>(v0, v1, cta_out);
  if (threadIdx.x == 0) { partC[2 * c] = cta_out[0]; partC[2 * c + 1] = cta_out[1]; }
  const bool go = grid_barrier(a.S, (unsigned)G, a.budget);
  grid_partials2(partC, G, bc);
  double rz = bc[0];
  const double bb = bc[1];
  const double tol2 = a.tol * a.tol * bb;
  double rr = bb;
  int it = 0;
  bool done = !go || !(bb > 0);
  while (!done) {
    // ---- A: Ap = S p by chunks, then per row in chunk order; partial p.Ap
    for (int q = q0 + warp; q < q1; q += NW) {
      DotAcc<T> acc[6];
      if (SOA) {
        const int blk = a.chunk_beg[q] + lane;
        T B[36];
        load_block36(a.Sval + s_idx(blk, 0), B);
        spmv_block(B, a, a.col[blk], acc);
      } else {
        const int e = a.chunk_beg[q + 1];
        for (int blk = a.chunk_beg[q] + lane; blk < e; blk += 32) {
          const T* B = a.Sval + (size_t)blk * BS2;
          const double* pb = a.p + 6 * (size_t)a.col[blk];
          double xv[6];
#pragma unroll
          for (int j = 0; j < 6; ++j) xv[j] = __ldcg(&pb[j]);
          block_dot6(B, xv, acc);
        }
      }
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        const DotAcc<T> y = warp_sum_acc(acc[i]);
        if (lane == 0) chunk_y[6 * (q - q0) + i] = y;
      }
    }
    __syncthreads();
    double pap = 0;
    for (int row = r0 + threadIdx.x; row < r1; row += NT) {
      DotAcc<T> y[6];
      for (int q = a.row_chunk0[row]; q < a.row_chunk0[row + 1]; ++q)
#pragma unroll
        for (int i = 0; i < 6; ++i) acc_add(y[i], chunk_y[6 * (q - q0) + i]);
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        const double yv = y[i].value();
        a.Ap[6 * row + i] = yv;
        pap += yv * a.p[6 * row + i];
      }
    }
    cta_sum2<NT>(pap, 0.0, cta_out);
    if (threadIdx.x == 0) { partA[2 * c] = cta_out[0]; partA[2 * c + 1] = 0; }
    if (!grid_barrier(a.S, (unsigned)G, a.budget)) break;
    grid_partials2(partA, G, bc);
    const double alpha = rz / bc[0];
    // ---- B: x += alpha p, r -= alpha Ap, z = M^-1 r; partial r.r, r.z
    v0 = 0; v1 = 0;
    for (int row = r0 + threadIdx.x; row < r1; row += NT) {
      double rv[6], zv[6];
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        a.x[6 * row + i] += alpha * a.p[6 * row + i];
        rv[i] = a.r[6 * row + i] - alpha * a.Ap[6 * row + i];
        a.r[6 * row + i] = rv[i];
      }
      apply_block(a.Minv + (size_t)row * BS2, rv, zv);
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        a.z[6 * row + i] = zv[i];
        v0 += rv[i] * rv[i];
        v1 += rv[i] * zv[i];
      }
    }
    cta_sum2<NT>(v0, v1, cta_out);
    if (threadIdx.x == 0) { partB[2 * c] = cta_out[0]; partB[2 * c + 1] = cta_out[1]; }
    if (!grid_barrier(a.S, (unsigned)G, a.budget)) break;
    grid_partials2(partB, G, bc);
    rr = bc[0];
    const double rz_new = bc[1];
    ++it;
    if (rr <= tol2 || it >= a.max_iters || !(rr == rr)) break;
    const double beta = rz_new / rz;
    rz = rz_new;
    // ---- C: p = z + beta p
    for (int k = 6 * r0 + threadIdx.x; k < 6 * r1; k += NT) {
      const double pk = a.z[k] + beta * a.p[k];
      a.p[k] = pk;
      if (a.phl) a.phl[k] = split2(pk);
    }
    if (!grid_barrier(a.S, (unsigned)G, a.budget)) break;
  }
  if (c == 0 && threadIdx.x == 0) {
    a.S->iters = it;
    a.S->rr = rr;
    a.S->bnorm2 = bb;
    a.S->rz = rz;
    a.S->done = 1;
  }
}

// ----------------------------------------------------------------------------
// Grid path of K5/K6: S streamed by the Tensor Memory Accelerator, CG in the Chronopoulos-Gear form.
//
// A CTA multiplies a contiguous run of 32-block chunks of the padded storage (one chunk = 32 whole blocks,
// 4.6 KB in float), the runs of about equal weight whatever the row lengths: a long row (a plane or a
// vanishing point seen by many cameras) may be cut between CTAs.  A row belongs to the CTA holding its first
// chunk, which updates its vector entries; a CTA whose run starts inside a row it does not own leaves its
// partial product of that row in a carry slot, added by the owner after the grid barrier that follows the
// product (the partial dot (w, u) needs no carry: it is a sum over the pieces).  The run is split into NW
// contiguous pieces, one per warp; a warp keeps NBUF chunks of its piece in flight in shared memory, each fetched by two
// bulk copies (cp.async.bulk: the values and the 32 column indices, completion counted on an mbarrier
// per buffer), so the stream of S never waits on the products.  Every wait on an mbarrier is bounded: if a copy has not landed after a very long
// spin the kernel records PCG_FLAG_TIMEOUT, finishes the iteration and stops; the host then returns
// BA_ERR_TIMEOUT.
//
// CG in the Chronopoulos-Gear form (one fused reduction per iteration) needs two grid barriers per
// iteration instead of three: u = M^-1 r must be complete before w = S u, and the partial dots
// (r, u), (r, r) and (w, u) must be complete before alpha and beta.  With s = S p carried as a vector:
//   x += alpha p;  r -= alpha s;  u = M^-1 r;  w = S u;  gamma' = (r, u);  delta = (w, u)
//   beta = gamma' / gamma;  alpha = gamma' / (delta - beta gamma' / alpha);  p = u + beta p;  s = w + beta s
// which produces the iterates of the standard preconditioned CG (the oracle's) in exact arithmetic.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
// the same copy with an L2 eviction-priority policy (createpolicy)
__device__ __forceinline__ void bulk_g2s_hint(void* dst, const void* src, unsigned bytes, uint64_t* bar, uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;\n" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
      : "memory");
}
__device__ __forceinline__ uint64_t l2_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;\n" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t l2_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(p));
  return p;
}
// true once the barrier's phase with the given parity has completed; false after `limit` polls
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, int limit) {
  const unsigned a = smem_u32(bar);
  for (int i = 0; i < limit; ++i) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

template <class T>
struct PcgStreamArgs {
  int64_t na;
  const int32_t *col, *row_chunk0, *chunk_beg;
  const int4* cta_part;   // per CTA {q0, q1, t0, t1}: chunks [q0, q1), touched block rows [t0, t1)
  double* carry;          // per CTA: its partial w of its first row when another CTA owns that row
  const T *Sval, *Minv;
  const double* b;
  double *x, *r, *u, *p, *w, *s;
  float2* uhl;   // float working type: u split into (hi, lo) floats for the products
  double* part;  // per-CTA partial sums, two parity slots of 3 x G
  DevScalars* S;
  double tol;
  int max_iters;
  float keep_frac;   // fraction of every warp's chunks fetched with L2 evict_last (kept across iterations)
  long long budget;  // clock64 cycles a grid barrier may wait
};

template <class T>
struct StreamCfg;
template <>
struct StreamCfg<float> { static constexpr int NT = 256, NBUF = 4; };
template <>
struct StreamCfg<double> { static constexpr int NT = 256, NBUF = 2; };
template <class T>
constexpr size_t stream_chunk_bytes() { return (size_t)BS2 * 32 * sizeof(T); }
template <class T>
constexpr size_t stream_stage_bytes() { return (size_t)(StreamCfg<T>::NT / 32) * StreamCfg<T>::NBUF * stream_chunk_bytes<T>(); }

// the u block a lane multiplies: the pre-split (hi, lo) floats (float S), or the FP64 values
template <class T>
struct UVal;
template <>
struct UVal<float> {
  float xh[6], xl[6];
  __device__ __forceinline__ void gather(const PcgStreamArgs<float>& a, int col) {
    // three 16-byte loads: the vector is 256-byte aligned and a block row starts on a 48-byte boundary
    const float4* pb = reinterpret_cast<const float4*>(a.uhl + 6 * (size_t)col);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const float4 v = __ldcg(&pb[j]);
      xh[2 * j] = v.x;
      xl[2 * j] = v.y;
      xh[2 * j + 1] = v.z;
      xl[2 * j + 1] = v.w;
    }
  }
  __device__ __forceinline__ void product(const float (&B)[36], DotAcc<float> (&acc)[6]) const {
    block_dot6_split(B, xh, xl, acc);
  }
};
template <>
struct UVal<double> {
  double xv[6];
  __device__ __forceinline__ void gather(const PcgStreamArgs<double>& a, int col) {
    const double2* pb = reinterpret_cast<const double2*>(a.u + 6 * (size_t)col);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const double2 v = __ldcg(&pb[j]);
      xv[2 * j] = v.x;
      xv[2 * j + 1] = v.y;
    }
  }
  __device__ __forceinline__ void product(const double (&B)[36], DotAcc<double> (&acc)[6]) const {
    block_dot6(B, xv, acc);
  }
};

template <class T, int NT, int NBUF>
__global__ void __launch_bounds__(NT, 1) k_pcg_stream(PcgStreamArgs<T> a) {
  constexpr int NW = NT / 32;
  constexpr unsigned CHB = (unsigned)stream_chunk_bytes<T>();
  constexpr int SPIN = 1 << 22;
  extern __shared__ __align__(128) unsigned char dyn[];
  T* stage = reinterpret_cast<T*>(dyn);                                          // [NW][NBUF][32 blocks x 36]
  DotAcc<T>* seg = reinterpret_cast<DotAcc<T>*>(dyn + stream_stage_bytes<T>());  // [row segments][6]
  __shared__ __align__(8) uint64_t bars[NW][NBUF];
  __shared__ __align__(128) int cols[NW][NBUF][32];
  __shared__ int wfirst[NW], wlast[NW], wbase[NW + 1];
  __shared__ double bc[4];
  __shared__ double cta_out[2];
  __shared__ double red3[NW][3];
  const int G = gridDim.x, c = blockIdx.x;
  const int4 pc = a.cta_part[c];
  const int q0 = pc.x, q1 = pc.y;   // chunks [q0, q1)
  const int r0 = pc.z, r1 = pc.w;   // block rows touched [r0, r1)
  const int o0 = (r0 < r1 && a.row_chunk0[r0] != q0) ? r0 + 1 : r0;   // block rows owned [o0, r1)
  const bool tail_cut = o0 < r1 && a.row_chunk0[r1] > q1;            // the last owned row continues
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // warp w multiplies the contiguous chunks [c0, c1) of the CTA's run; a lane accumulates its block
  // position over all chunks of one block row and the warp sums the lanes once per row it touches,
  // leaving one "row segment" (6 sums) per (warp, row)
  const int ntot = q1 - q0;
  const int c0 = q0 + (int)((int64_t)ntot * warp / NW), c1 = q0 + (int)((int64_t)ntot * (warp + 1) / NW);
  const int nk = c1 - c0;
  // S does not fit in L2: the first keep_frac of the warp's chunks are fetched evict_last so that they stay
  // resident from one iteration to the next, the rest evict_first so that they do not displace them
  const int nkeep = (int)((float)nk * a.keep_frac);
  const uint64_t pol_keep = l2_evict_last(), pol_stream = l2_evict_first();
  auto row_of = [&](int q) {   // the block row holding chunk q (r0 <= row < r1)
    int lo = r0, hi = r1 - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (a.row_chunk0[mid] <= q) lo = mid; else hi = mid - 1;
    }
    return lo;
  };
  if (lane == 0) {
    for (int bi = 0; bi < NBUF; ++bi) mbar_init(&bars[warp][bi], 1);
    wfirst[warp] = nk > 0 ? row_of(c0) : 0;
    wlast[warp] = nk > 0 ? row_of(c1 - 1) : -1;
  }
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0) {
    int b = 0;
    for (int w = 0; w < NW; ++w) { wbase[w] = b; b += wlast[w] - wfirst[w] + 1; }
    wbase[NW] = b;
  }
  __syncthreads();
  unsigned phase = 0;   // bit bi: parity of the next completion of buffer bi
  bool timed_out = false;
  bool prefetched = false;   // the first NBUF chunks of the next product are already in flight

  // w = S u over this CTA's rows; returns (w, u) over the CTA's rows.  Software pipeline per warp: the
  // values and column indices of chunk k + NBUF are in flight (TMA) while chunk k is multiplied, and the
  // u values of chunk k + 1 are gathered (L2) before the products of chunk k are formed.
  auto spmv = [&](double& wu) {
    auto issue = [&](int k) {
      const int q = c0 + k;
      const int bi = k % NBUF;
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      mbar_expect_tx(&bars[warp][bi], CHB + 128u);
      const uint64_t pol = k < nkeep ? pol_keep : pol_stream;
      bulk_g2s_hint(stage + ((size_t)warp * NBUF + bi) * (BS2 * 32), a.Sval + s_idx(a.chunk_beg[q], 0), CHB,
                    &bars[warp][bi], pol);
      bulk_g2s_hint(&cols[warp][bi][0], a.col + a.chunk_beg[q], 128u, &bars[warp][bi], pol);
    };
    auto arrive = [&](int k) {   // wait for chunk k's copies
      const int bi = k % NBUF;
      if (!mbar_wait(&bars[warp][bi], (phase >> bi) & 1u, SPIN)) timed_out = true;
      phase ^= 1u << bi;
    };
    if (lane == 0 && !prefetched)
      for (int k = 0; k < NBUF && k < nk; ++k) issue(k);
    prefetched = false;
    DotAcc<T> acc[6];
    int row = wfirst[warp];
    int rend = nk > 0 ? a.row_chunk0[row + 1] : 0;
    auto flush = [&]() {   // the warp's sums of `row` into its segment, then a fresh accumulator
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        const DotAcc<T> y = warp_sum_acc(acc[i]);
        if (lane == 0) seg[6 * (wbase[warp] + row - wfirst[warp]) + i] = y;
        acc[i] = DotAcc<T>();
      }
    };
    UVal<T> un;   // u of this lane's column in the next chunk
    if (nk > 0) {
      arrive(0);
      un.gather(a, cols[warp][0][lane]);
    }
    for (int k = 0; k < nk; ++k) {
      const int q = c0 + k;
      while (q >= rend) {
        flush();
        ++row;
        rend = a.row_chunk0[row + 1];
      }
      const int bi = k % NBUF;
      T B[36];
      load_block36(stage + ((size_t)warp * NBUF + bi) * (BS2 * 32) + lane * 36, B);
      const UVal<T> uc = un;
      if (k + 1 < nk) {
        arrive(k + 1);
        un.gather(a, cols[warp][(k + 1) % NBUF][lane]);
      }
      __syncwarp();   // every lane holds its block: the buffer may be refilled while the products run
      if (lane == 0 && k + NBUF < nk) issue(k + NBUF);
      uc.product(B, acc);
    }
    if (nk > 0) flush();
    // S is the same in every iteration: start the next product's first chunks now, so that they stream
    // in while the vectors are updated and the grid waits at its barriers
    __syncwarp();
    if (lane == 0)
      for (int k = 0; k < NBUF && k < nk; ++k) issue(k);
    prefetched = true;
    __syncthreads();
    double v = 0;
    for (int r = r0 + threadIdx.x; r < r1; r += NT) {
      DotAcc<T> y[6];
      for (int w = 0; w < NW; ++w)
        if (wfirst[w] <= r && r <= wlast[w])
#pragma unroll
          for (int i = 0; i < 6; ++i) acc_add(y[i], seg[6 * (wbase[w] + r - wfirst[w]) + i]);
      double* dst = r < o0 ? a.carry + 6 * (size_t)c : a.w + 6 * (size_t)r;
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        const double yv = y[i].value();
        dst[i] = yv;
        v += yv * __ldcg(&a.u[6 * r + i]);   // u of a row owned by another CTA: not through L1
      }
    }
    wu = v;
  };
  // u = M^-1 r for the CTA's rows (and its split copy); partial (r, u) and (r, r)
  auto drain = [&]() {   // wait for prefetched copies before the kernel ends
    if (!prefetched) return;
    for (int k = 0; k < NBUF && k < nk; ++k) {
      const int bi = k % NBUF;
      if (!mbar_wait(&bars[warp][bi], (phase >> bi) & 1u, SPIN)) timed_out = true;
      phase ^= 1u << bi;
    }
    prefetched = false;
  };
  // after the grid barrier that follows a product: the partial sums of the last owned row left by the
  // following CTAs (every CTA whose run starts inside that row)
  auto add_carries = [&]() {
    if (!tail_cut || threadIdx.x >= 6) return;
    const int row = r1 - 1;
    double v = a.w[6 * (size_t)row + threadIdx.x];
    for (int c2 = c + 1; c2 < G; ++c2) {
      const int4 pn = a.cta_part[c2];
      if (pn.x == pn.y || pn.z != row) break;
      v += __ldcg(&a.carry[6 * (size_t)c2 + threadIdx.x]);
    }
    a.w[6 * (size_t)row + threadIdx.x] = v;
  };
  auto precondition = [&](double& ru, double& rr_) {
    double v0 = 0, v1 = 0;
    for (int k = o0 * 6 + threadIdx.x; k < r1 * 6; k += NT) {   // one output per thread
      const int row = k / 6, i = k - 6 * row;
      const T* M = a.Minv + (size_t)row * BS2 + 6 * i;
      const double* rv = a.r + 6 * (size_t)row;
      T zs = 0;
#pragma unroll
      for (int j = 0; j < 6; ++j) zs += M[j] * (T)rv[j];
      const double z = (double)zs, ri = rv[i];
      a.u[k] = z;
      if (a.uhl) a.uhl[k] = split2(z);
      v0 += ri * z;
      v1 += ri * ri;
    }
    ru = v0;
    rr_ = v1;
  };
  auto slot = [&](int par, int k) { return a.part + (size_t)par * 3 * G + (size_t)k * G; };

  // ---- start: x = 0, r = b, u = M^-1 r, w = S u
  for (int k = o0 * 6 + threadIdx.x; k < r1 * 6; k += NT) { a.x[k] = 0; a.r[k] = a.b[k]; }
  __syncthreads();
  double ru, rrl, wu;
  precondition(ru, rrl);
  cta_sum2<NT>(ru, rrl, cta_out);
  if (threadIdx.x == 0) { slot(0, 0)[c] = cta_out[0]; slot(0, 1)[c] = cta_out[1]; }
  // a copy wait that ran out (in any warp) is recorded before the barrier; the barrier's answer is uniform
  unsigned long long bar_target = 0;   // arrivals that complete this CTA's next barrier
  auto sync = [&]() -> bool {
    if (timed_out) atomicOr(&a.S->flags, PCG_FLAG_TIMEOUT);
    bar_target += (unsigned long long)G;
    return grid_barrier_count(a.S, bar_target, timed_out, a.budget);
  };
  bool go = sync();
  if (go) {
    spmv(wu);
    cta_sum2<NT>(wu, 0.0, cta_out);
    if (threadIdx.x == 0) slot(0, 2)[c] = cta_out[0];
    go = sync();
  }
  if (go) add_carries();   // ordered before the vector updates by the barriers inside reduce3
  auto reduce3 = [&](int par) {   // the three global sums, formed identically in every CTA
    double s0 = 0, s1 = 0, s2 = 0;
    for (int g = threadIdx.x; g < G; g += NT) {
      s0 += __ldcg(&slot(par, 0)[g]);
      s1 += __ldcg(&slot(par, 1)[g]);
      s2 += __ldcg(&slot(par, 2)[g]);
    }
    s0 = warp_sum(s0);
    s1 = warp_sum(s1);
    s2 = warp_sum(s2);
    if (lane == 0) { red3[warp][0] = s0; red3[warp][1] = s1; red3[warp][2] = s2; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double t0 = 0, t1 = 0, t2 = 0;
      for (int w = 0; w < NW; ++w) { t0 += red3[w][0]; t1 += red3[w][1]; t2 += red3[w][2]; }
      bc[0] = t0; bc[1] = t1; bc[2] = t2;
    }
    __syncthreads();
  };
  if (go) reduce3(0);
  double gam = go ? bc[0] : 0.0;
  const double bb = go ? bc[1] : 0.0;
  double alpha = go && bc[2] > 0 ? gam / bc[2] : 0.0;
  const double tol2 = a.tol * a.tol * bb;
  double rr = bb;
  int it = 0;
  bool done = !go || !(bb > 0) || !(bc[2] > 0);
  double beta = 0;
  int par = 1;
  while (!done) {
    // p = u + beta p, s = w + beta s (p = u, s = w on the first pass: p and s hold no values yet),
    // x += alpha p, r -= alpha s; then u = M^-1 r; partial (r, u), (r, r)
    const bool first = it == 0;
    for (int k = o0 * 6 + threadIdx.x; k < r1 * 6; k += NT) {
      const double pk = first ? a.u[k] : a.u[k] + beta * a.p[k];
      const double sk = first ? a.w[k] : a.w[k] + beta * a.s[k];
      a.p[k] = pk;
      a.s[k] = sk;
      a.x[k] += alpha * pk;
      a.r[k] -= alpha * sk;
    }
    __syncthreads();
    precondition(ru, rrl);
    cta_sum2<NT>(ru, rrl, cta_out);
    if (threadIdx.x == 0) { slot(par, 0)[c] = cta_out[0]; slot(par, 1)[c] = cta_out[1]; }
    ++it;
    if (!sync()) break;
    spmv(wu);
    cta_sum2<NT>(wu, 0.0, cta_out);
    if (threadIdx.x == 0) slot(par, 2)[c] = cta_out[0];
    if (!sync()) break;
    add_carries();
    reduce3(par);
    const double gam_new = bc[0], delta = bc[2];
    rr = bc[1];
    if (rr <= tol2 || it >= a.max_iters || !(rr == rr)) break;
    beta = gam_new / gam;
    const double den = delta - beta * gam_new / alpha;
    alpha = gam_new / den;
    gam = gam_new;
    if (!(den > 0)) break;   // S not positive definite along p (rounding): keep the current x
    par ^= 1;
  }
  drain();
  if (timed_out) atomicOr(&a.S->flags, PCG_FLAG_TIMEOUT);
  if (c == 0 && threadIdx.x == 0) {
    a.S->iters = it;
    a.S->rr = rr;
    a.S->bnorm2 = bb;
    a.S->rz = gam;
    a.S->done = 1;
  }
}

// ============================================================================
// K5/K6 on the typed storage: camera rows stream their camera-camera, camera-plane and camera-VP chunks;
// every camera-group block also adds its transpose times the camera's u to the group's values
// (a per-warp shared-memory accumulator: the blocks of one chunk lie in one camera row and so name
// distinct groups), and the CTAs' group partials are summed in CTA order after the grid barrier.
// ============================================================================
template <class T>
struct PcgTypedArgs {
  int64_t na, nc, npl, nv;
  int gv;                         // group values: 3 per plane, 2 per VP
  const int32_t *tcol, *row_chunk0, *gg_ptr, *gg_col, *cta_gs, *gv_idx;
  const int4* tchunk;             // per chunk {value offset, first block, camera row, type}
  const int4* cta_part;           // per CTA {q0, q1, t0, t1} over the camera rows' chunks
  double* carry;                  // per CTA: its partial w of its first camera row when another CTA owns it
  double* part_g;                 // per group value, every CTA's scatter into it (gv x G)
  const T *Sv, *Minv;
  int64_t gg_val0;                // first value of the group-group blocks in Sv
  const double* b;
  double *x, *r, *u, *p, *w, *s;
  float2* uhl;                    // float working type: u split into (hi, lo) floats
  double* part;                   // per-CTA partial sums, two parity slots of 3 x G
  DevScalars* S;
  double tol;
  int max_iters;
  float keep_frac;
  long long budget;
  int nown;                       // shared-memory room for the owned values (the most any CTA owns)
};

// one operand value: the (hi, lo) split of an FP64 value for float S, the value itself for double S
template <class T>
struct XV;
template <>
struct XV<float> {
  float h, l;
  __device__ __forceinline__ void set(const float2 v) { h = v.x; l = v.y; }
};
template <>
struct XV<double> {
  double v;
};
// acc += b * x: for float a double-single step (exact product by FMA, TwoSum into the running sum,
// the same operations as block_dot6_split); for double one FMA
__device__ __forceinline__ void ds_madd(DotAcc<float>& a, float b, const XV<float>& x) {
  const float ph = b * x.h;
  const float pe = fmaf(b, x.h, -ph);
  const float sm = a.hi + ph;
  const float bp = sm - a.hi;
  const float err = (a.hi - (sm - bp)) + (ph - bp);
  a.hi = sm;
  a.lo += err + fmaf(b, x.l, pe);
}
__device__ __forceinline__ void ds_madd(DotAcc<float>& a, float b, const XV<float>& x);
__device__ __forceinline__ void ds_madd(DotAcc<double>& a, double b, const XV<double>& x) { a.s = fma(b, x.v, a.s); }
// acc += sum_j b[j * bs] x[j] over N terms of one stored block: for float the block's short dot product in
// float FMA (head and tail parts of x; its rounding is a few units of the block's own float entries, the
// order of their storage rounding) added to the double-single sum once; for double plain FMA
template <int N>
__device__ __forceinline__ void blk_dot(DotAcc<float>& acc, const float* b, int bs, const XV<float>* x) {
  float h = 0.f, l = 0.f;
#pragma unroll
  for (int j = 0; j < N; ++j) { h = fmaf(b[j * bs], x[j].h, h); l = fmaf(b[j * bs], x[j].l, l); }
  two_sum_acc(acc.hi, acc.lo, h, l);
}
template <int N>
__device__ __forceinline__ void blk_dot(DotAcc<double>& acc, const double* b, int bs, const XV<double>* x) {
#pragma unroll
  for (int j = 0; j < N; ++j) acc.s = fma(b[j * bs], x[j].v, acc.s);
}

// the 6 values of block row r in three 16-byte loads (every vector starts on a 256-byte boundary and a block row
// on a 48-byte one): half the L2 sector requests of six 8-byte gathers
__device__ __forceinline__ void load_xv6(const PcgTypedArgs<float>& a, size_t r, XV<float> (&x)[6]) {
  const float4* q = reinterpret_cast<const float4*>(a.uhl + 6 * r);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float4 t = __ldcg(q + k);
    x[2 * k].h = t.x; x[2 * k].l = t.y; x[2 * k + 1].h = t.z; x[2 * k + 1].l = t.w;
  }
}
__device__ __forceinline__ void load_xv6(const PcgTypedArgs<double>& a, size_t r, XV<double> (&x)[6]) {
  const double2* q = reinterpret_cast<const double2*>(a.u + 6 * r);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double2 t = __ldcg(q + k);
    x[2 * k].v = t.x; x[2 * k + 1].v = t.y;
  }
}

// n contiguous values of a lane's block from the stage buffer (16-byte aligned for 36 and 12 floats and for
// every double block; 8-byte aligned for 18 floats)
template <int N>
__device__ __forceinline__ void load_vals(const float* p, float (&B)[N]) {
  if constexpr (N % 4 == 0) {
    const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int k = 0; k < N / 4; ++k) {
      const float4 t = q[k];
      B[4 * k] = t.x; B[4 * k + 1] = t.y; B[4 * k + 2] = t.z; B[4 * k + 3] = t.w;
    }
  } else {
    const float2* q = reinterpret_cast<const float2*>(p);
#pragma unroll
    for (int k = 0; k < N / 2; ++k) {
      const float2 t = q[k];
      B[2 * k] = t.x; B[2 * k + 1] = t.y;
    }
  }
}
template <int N>
__device__ __forceinline__ void load_vals(const double* p, double (&B)[N]) {
  const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
  for (int k = 0; k < N / 2; ++k) {
    const double2 t = q[k];
    B[2 * k] = t.x; B[2 * k + 1] = t.y;
  }
}

template <class T>
struct TypedCfg;
template <>
struct TypedCfg<float> { static constexpr int NT = 256, NBUF = 3; };
template <>
struct TypedCfg<double> { static constexpr int NT = 128, NBUF = 4; };
template <class T>
constexpr size_t typed_stage_bytes() {
  return (size_t)(TypedCfg<T>::NT / 32) * TypedCfg<T>::NBUF * TCHUNK * 36 * sizeof(T);
}
// the operand copy of the group values in shared memory
template <class T>
using UGv = typename std::conditional<sizeof(T) == 4, float2, double>::type;
// dynamic shared memory: stage | per-warp group accumulators | group operand values | camera-row segments
template <class T>
__host__ __device__ constexpr size_t typed_gvp(int gv) { return (size_t)((gv + GV_PAD + 1) & ~1); }
template <class T>
__host__ __device__ constexpr size_t typed_fixed_smem(int gv) {
  return typed_stage_bytes<T>() + (size_t)(TypedCfg<T>::NT / 32) * typed_gvp<T>(gv) * sizeof(DotAcc<T>) +
         typed_gvp<T>(gv) * sizeof(UGv<T>);
}

template <class T, int NT, int NBUF>
__global__ void __launch_bounds__(NT, 1) k_pcg_typed(PcgTypedArgs<T> a) {
  constexpr int NW = NT / 32;
  constexpr int SPIN = 1 << 22;   // polls of a bulk copy's completion (the copies always complete)
  extern __shared__ __align__(128) unsigned char dyn[];
  const int gvp = (int)typed_gvp<T>(a.gv);
  T* stage = reinterpret_cast<T*>(dyn);                                                    // [NW][NBUF][32 x 36]
  DotAcc<T>* gacc = reinterpret_cast<DotAcc<T>*>(dyn + typed_stage_bytes<T>());           // [NW][gvp]
  UGv<T>* ug = reinterpret_cast<UGv<T>*>(reinterpret_cast<unsigned char*>(gacc) + sizeof(DotAcc<T>) * NW * gvp);
  // the owned values' vectors stay in shared memory across iterations: x, r, p, s, w, u (double) and the
  // owned block rows' block-Jacobi inverses (36 per row); only u (which every CTA gathers), the carries and the
  // group scatter go through global memory
  double* sv = reinterpret_cast<double*>(dyn + typed_fixed_smem<T>(a.gv));
  double *sx = sv, *sr = sv + a.nown, *sp = sv + 2 * a.nown, *ss = sv + 3 * a.nown, *sw = sv + 4 * a.nown,
         *su = sv + 5 * a.nown;
  T* sM = reinterpret_cast<T*>(sv + 6 * a.nown);                                           // [owned rows][36]
  DotAcc<T>* seg = reinterpret_cast<DotAcc<T>*>(
      reinterpret_cast<unsigned char*>(sM) + ((sizeof(T) * 6 * (size_t)a.nown + 15) & ~(size_t)15));   // [row segments][6]
  __shared__ __align__(8) uint64_t bars[NW][NBUF];
  __shared__ __align__(128) int cols[NW][NBUF][TCHUNK];
  __shared__ int wfirst[NW], wlast[NW], wbase[NW + 1];
  __shared__ double bc[4];
  __shared__ double cta_out[2];
  __shared__ double red3[NW][3];
  const int G = gridDim.x, c = blockIdx.x;
  const int4 pc = a.cta_part[c];
  const int q0 = pc.x, q1 = pc.y;   // chunks [q0, q1)
  const int r0 = pc.z, r1 = pc.w;   // camera rows touched [r0, r1)
  const int o0 = (r0 < r1 && a.row_chunk0[r0] != q0) ? r0 + 1 : r0;   // camera rows owned [o0, r1)
  const bool tail_cut = o0 < r1 && a.row_chunk0[r1] > q1;            // the last owned row continues
  const int gs0 = a.cta_gs[c], gs1 = a.cta_gs[c + 1];                 // group rows owned [gs0, gs1)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntot = q1 - q0;
  const int c0 = q0 + (int)((int64_t)ntot * warp / NW), c1 = q0 + (int)((int64_t)ntot * (warp + 1) / NW);
  const int nk = c1 - c0;
  const int nkeep = (int)((float)nk * a.keep_frac);
  const uint64_t pol_keep = l2_evict_last(), pol_stream = l2_evict_first();
  DotAcc<T>* ga = gacc + (size_t)warp * gvp;
  auto row_of = [&](int q) {
    int lo = r0, hi = r1 - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (a.row_chunk0[mid] <= q) lo = mid; else hi = mid - 1;
    }
    return lo;
  };
  if (lane == 0) {
    for (int bi = 0; bi < NBUF; ++bi) mbar_init(&bars[warp][bi], 1);
    wfirst[warp] = nk > 0 ? row_of(c0) : 0;
    wlast[warp] = nk > 0 ? row_of(c1 - 1) : -1;
  }
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0) {
    int b = 0;
    for (int w = 0; w < NW; ++w) { wbase[w] = b; b += wlast[w] - wfirst[w] + 1; }
    wbase[NW] = b;
  }
  __syncthreads();
  unsigned phase = 0;
  bool timed_out = false;
  bool prefetched = false;
  // the owned values: camera rows [o0, r1) and group rows [gs0, gs1) (6 per row)
  const int64_t cb0 = 6 * (int64_t)o0, cb1 = 6 * (int64_t)r1;
  const int64_t gb0 = 6 * (a.nc + gs0), gb1 = 6 * (a.nc + gs1);
  // f(global index, local index) over the owned values
  auto owned = [&](auto&& f) {
    for (int64_t k = cb0 + threadIdx.x; k < cb1; k += NT) f(k, (int)(k - cb0));
    for (int64_t k = gb0 + threadIdx.x; k < gb1; k += NT) f(k, (int)(cb1 - cb0 + k - gb0));
  };
  auto loc_cam = [&](int64_t k) { return (int)(k - cb0); };                 // an owned camera value
  auto loc_grp = [&](int64_t k) { return (int)(cb1 - cb0 + k - gb0); };     // an owned group value
  // group row g's group values: first value offset and count
  auto gval = [&](int g, int& k0, int& nd) {
    if (g < a.npl) { k0 = 3 * g; nd = 3; }
    else if (g < a.npl + a.nv) { k0 = 3 * (int)a.npl + 2 * (g - (int)a.npl); nd = 2; }
    else { k0 = 3 * (int)a.npl + 2 * (int)a.nv + 3 * (g - (int)(a.npl + a.nv)); nd = 3; }   // intrinsics
  };

  auto issue = [&](int k) {
    const int q = c0 + k;
    const int bi = k % NBUF;
    const int4 cd = __ldg(&a.tchunk[q]);
    const unsigned vb = (unsigned)(TCHUNK * ty_vals(cd.w) * sizeof(T));
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    mbar_expect_tx(&bars[warp][bi], vb + 4u * TCHUNK);
    const uint64_t pol = k < nkeep ? pol_keep : pol_stream;
    bulk_g2s_hint(stage + ((size_t)warp * NBUF + bi) * (TCHUNK * 36), a.Sv + cd.x, vb, &bars[warp][bi], pol);
    bulk_g2s_hint(&cols[warp][bi][0], a.tcol + cd.y, 4u * TCHUNK, &bars[warp][bi], pol);
  };
  auto arrive = [&](int k) {
    const int bi = k % NBUF;
    if (!mbar_wait(&bars[warp][bi], (phase >> bi) & 1u, SPIN)) timed_out = true;
    phase ^= 1u << bi;
  };
  auto drain = [&]() {
    if (!prefetched) return;
    for (int k = 0; k < NBUF && k < nk; ++k) arrive(k);
    prefetched = false;
  };

  // w = S u over the owned values (camera rows complete after the carries, group rows after the partials);
  // returns this CTA's share of (w, u)
  auto spmv = [&](double& wu) {
    // the group values of u, eight per thread at a time: the (read-only, L1-resident) indices, then the eight
    // gathers issued together, so that a thread waits for two round trips per eight values rather than two per value
    constexpr int UGB = 8;
    for (int k0 = threadIdx.x; k0 < gvp; k0 += UGB * NT) {
      int gi[UGB];
#pragma unroll
      for (int t = 0; t < UGB; ++t) {
        const int k = k0 + t * NT;
        gi[t] = k < a.gv ? __ldg(&a.gv_idx[k]) : -1;
      }
      UGv<T> gvv[UGB];
#pragma unroll
      for (int t = 0; t < UGB; ++t) {
        if constexpr (sizeof(T) == 4) gvv[t] = gi[t] >= 0 ? __ldcg(&a.uhl[gi[t]]) : make_float2(0.f, 0.f);
        else gvv[t] = gi[t] >= 0 ? __ldcg(&a.u[gi[t]]) : 0.0;
      }
#pragma unroll
      for (int t = 0; t < UGB; ++t)
        if (k0 + t * NT < gvp) ug[k0 + t * NT] = gvv[t];
    }
    for (int k = lane; k < gvp; k += 32) ga[k] = DotAcc<T>();
    if (lane == 0 && !prefetched)
      for (int k = 0; k < NBUF && k < nk; ++k) issue(k);
    prefetched = false;
    __syncthreads();
    DotAcc<T> acc[6];
    int row = wfirst[warp];
    int rend = nk > 0 ? __ldg(&a.row_chunk0[row + 1]) : 0;
    XV<T> ur[6];   // u of the current camera row
    auto load_ur = [&]() { load_xv6(a, (size_t)row, ur); };
    auto flush = [&]() {
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        const DotAcc<T> y = warp_sum_acc(acc[i]);
        if (lane == 0) seg[6 * (wbase[warp] + row - wfirst[warp]) + i] = y;
        acc[i] = DotAcc<T>();
      }
    };
    XV<T> un[6];   // u of this lane's column in the next camera-camera chunk
    int4 cdn = make_int4(0, 0, 0, -1);
    if (nk > 0) {
      load_ur();
      arrive(0);
      cdn = __ldg(&a.tchunk[c0]);
      if (cdn.w == TY_CC) {
        load_xv6(a, (size_t)cols[warp][0][lane], un);
      }
    }
    for (int k = 0; k < nk; ++k) {
      const int q = c0 + k;
      const int4 cd = cdn;
      while (q >= rend) {
        flush();
        ++row;
        rend = __ldg(&a.row_chunk0[row + 1]);
        load_ur();
      }
      const int bi = k % NBUF;
      const T* buf = stage + ((size_t)warp * NBUF + bi) * (TCHUNK * 36);
      const int col = cols[warp][bi][lane];
      // the lane's block into registers, then the next chunk's copies and gathers
      T B[36];
      XV<T> uc[6];
      if (cd.w == TY_CC) {
        load_block36(buf + lane * 36, B);
#pragma unroll
        for (int j = 0; j < 6; ++j) uc[j] = un[j];
      } else if (cd.w != TY_CV) {   // camera-plane or camera-intrinsics: 6 x 3
        T b18[18];
        load_vals<18>(buf + lane * 18, b18);
#pragma unroll
        for (int j = 0; j < 18; ++j) B[j] = b18[j];
      } else {
        T b12[12];
        load_vals<12>(buf + lane * 12, b12);
#pragma unroll
        for (int j = 0; j < 12; ++j) B[j] = b12[j];
      }
      // every lane holds its block and column: the buffer is refilled first, so that NBUF chunks are in
      // flight while the warp waits for the next one
      __syncwarp();
      if (lane == 0 && k + NBUF < nk) issue(k + NBUF);
      if (k + 1 < nk) {
        arrive(k + 1);
        cdn = __ldg(&a.tchunk[q + 1]);
        if (cdn.w == TY_CC) {
          load_xv6(a, (size_t)cols[warp][(k + 1) % NBUF][lane], un);
        }
      }
      if (cd.w == TY_CC) {
#pragma unroll
        for (int i = 0; i < 6; ++i) blk_dot<6>(acc[i], B + i * 6, 1, uc);
      } else {
        // camera-group block (6 x nd): the row part with the group's u, the transpose into the group values
        const int nd = cd.w == TY_CV ? 2 : 3;
        XV<T> xg[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          if (j < nd) {
            if constexpr (sizeof(T) == 4) xg[j].set(ug[col + j]); else xg[j].v = ug[col + j];
          }
        }
        if (nd == 3) {
#pragma unroll
          for (int i = 0; i < 6; ++i) blk_dot<3>(acc[i], B + i * 3, 1, xg);
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            DotAcc<T> y;
            blk_dot<6>(y, B + j, 3, ur);
            acc_add(ga[col + j], y);
          }
        } else {
#pragma unroll
          for (int i = 0; i < 6; ++i) blk_dot<2>(acc[i], B + i * 2, 1, xg);
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            DotAcc<T> y;
            blk_dot<6>(y, B + j, 2, ur);
            acc_add(ga[col + j], y);
          }
        }
      }
    }
    if (nk > 0) flush();
    __syncwarp();
    if (lane == 0)
      for (int k = 0; k < NBUF && k < nk; ++k) issue(k);
    prefetched = true;
    __syncthreads();
    double v = 0;
    // camera rows: the warps' segments, in warp order
    for (int rr = r0 + threadIdx.x; rr < r1; rr += NT) {
      DotAcc<T> y[6];
      for (int w = 0; w < NW; ++w)
        if (wfirst[w] <= rr && rr <= wlast[w])
#pragma unroll
          for (int i = 0; i < 6; ++i) acc_add(y[i], seg[6 * (wbase[w] + rr - wfirst[w]) + i]);
      if (rr < o0) {
#pragma unroll
        for (int i = 0; i < 6; ++i) {
          const double yv = y[i].value();
          a.carry[6 * (size_t)c + i] = yv;
          v += yv * __ldcg(&a.u[6 * (size_t)rr + i]);
        }
      } else {
        const int l0 = loc_cam(6 * (int64_t)rr);
#pragma unroll
        for (int i = 0; i < 6; ++i) {
          const double yv = y[i].value();
          sw[l0 + i] = yv;
          v += yv * su[l0 + i];
        }
      }
    }
    // the group values of this CTA's scatter, warps in order; their dot with u in the working precision
    // (the staged operand copy of u), rounded to double once
    DotAcc<T> vg;
    for (int k = threadIdx.x; k < a.gv; k += NT) {
      DotAcc<T> y = gacc[k];
      for (int w = 1; w < NW; ++w) acc_add(y, gacc[(size_t)w * gvp + k]);
      const double yv = y.value();
      a.part_g[(size_t)k * G + c] = yv;   // value-major: the group row's owner reads the CTAs' sums coalesced
      XV<T> uk;
      if constexpr (sizeof(T) == 4) uk.set(ug[k]); else uk.v = ug[k];
      if constexpr (sizeof(T) == 4) {
        // y u = (hi + lo)(u_hi + u_lo): the lo x lo term is below the working precision
        ds_madd(vg, y.hi, uk);
        XV<T> ul;
        ul.h = uk.h; ul.l = 0.f;
        ds_madd(vg, y.lo, ul);
      } else {
        ds_madd(vg, (T)yv, uk);
      }
    }
    v += vg.value();
    // the group-group blocks of the owned group rows (a VP parallel to many planes has a long row): a thread
    // per block, its 6 products into the group accumulators' space (free until the next product), then
    // every row's blocks summed in block order
    __syncthreads();
    DotAcc<T>* ggy = gacc;
    const int kb0 = __ldg(&a.gg_ptr[gs0]), kb1 = __ldg(&a.gg_ptr[gs1]);
    for (int kb = kb0 + threadIdx.x; kb < kb1; kb += NT) {
      T Bk[36];
      load_block36(a.Sv + a.gg_val0 + 36 * (size_t)kb, Bk);   // 16-byte aligned: gg_val0 is a chunk boundary
      const int cl = __ldg(&a.gg_col[kb]);
      XV<T> uv[6];
      load_xv6(a, (size_t)cl, uv);
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        DotAcc<T> y;
#pragma unroll
        for (int j = 0; j < 6; ++j) ds_madd(y, Bk[6 * i + j], uv[j]);
        ggy[6 * (size_t)(kb - kb0) + i] = y;
      }
    }
    __syncthreads();
    // a warp per owned group row: its lanes over the row's blocks in the working precision, then the
    // warp's shuffle tree
    for (int g = gs0 + warp; g < gs1; g += NW) {
      DotAcc<T> y[6];
      for (int kb = a.gg_ptr[g] + lane; kb < a.gg_ptr[g + 1]; kb += 32)
#pragma unroll
        for (int i = 0; i < 6; ++i) acc_add(y[i], ggy[6 * (size_t)(kb - kb0) + i]);
#pragma unroll
      for (int i = 0; i < 6; ++i) y[i] = warp_sum_acc(y[i]);
      if (lane == 0) {
#pragma unroll
        for (int i = 0; i < 6; ++i) {
          const int l = loc_grp(6 * ((int64_t)a.nc + g) + i);
          const double yv = y[i].value();
          sw[l] = yv;
          v += yv * su[l];
        }
      }
    }
    wu = v;
  };
  // after the grid barrier that follows a product: the carries of the last owned camera row, and the group
  // rows' sums of every CTA's scatter (in CTA order)
  auto add_carries = [&]() {
    if (tail_cut && threadIdx.x < 6) {
      const int rrow = r1 - 1;
      const int l = loc_cam(6 * (int64_t)rrow + threadIdx.x);
      double v = sw[l];
      for (int c2 = c + 1; c2 < G; ++c2) {
        const int4 pn = __ldg(&a.cta_part[c2]);
        if (pn.x == pn.y || pn.z != rrow) break;
        v += __ldcg(&a.carry[6 * (size_t)c2 + threadIdx.x]);
      }
      sw[l] = v;
    }
    // a warp per owned group value, its lanes over the CTAs (a fixed order: strided lane sums, then the
    // warp's shuffle tree)
    for (int t = warp; t < 3 * (gs1 - gs0); t += NW) {
      const int g = gs0 + t / 3, d = t % 3;
      int k0, nd;
      gval(g, k0, nd);
      if (d >= nd) continue;
      // the lane's CTAs in batches of eight loads issued together, summed in CTA order
      constexpr int CB = 8;
      const double* pg = a.part_g + (size_t)(k0 + d) * G;
      double v = 0;
      for (int cb = lane; cb < G; cb += CB * 32) {
        double pv[CB];
#pragma unroll
        for (int t = 0; t < CB; ++t) pv[t] = cb + 32 * t < G ? __ldcg(&pg[cb + 32 * t]) : 0.0;
#pragma unroll
        for (int t = 0; t < CB; ++t) v += pv[t];
      }
      v = warp_sum(v);
      if (lane == 0) sw[loc_grp(6 * ((int64_t)a.nc + g) + d)] += v;
    }
  };
  auto precondition = [&](double& ru, double& rr_) {
    double v0 = 0, v1 = 0;
    owned([&](int64_t k, int l) {
      const int i = (int)(k % 6);
      const T* M = sM + 6 * (size_t)l;        // row i of the block (the owned rows are whole)
      const double* rv = sr + (l - i);
      T zs = 0;
#pragma unroll
      for (int j = 0; j < 6; ++j) zs += M[j] * (T)rv[j];
      const double z = (double)zs, ri = rv[i];
      su[l] = z;
      a.u[k] = z;
      if (a.uhl) a.uhl[k] = split2(z);
      v0 += ri * z;
      v1 += ri * ri;
    });
    ru = v0;
    rr_ = v1;
  };
  auto slot = [&](int par, int k) { return a.part + (size_t)par * 3 * G + (size_t)k * G; };
  // a copy wait that ran out (in any warp) is recorded before the barrier; the barrier's answer is uniform
  unsigned long long bar_target = 0;   // arrivals that complete this CTA's next barrier
  auto sync = [&]() -> bool {
    if (timed_out) atomicOr(&a.S->flags, PCG_FLAG_TIMEOUT);
    bar_target += (unsigned long long)G;
    return grid_barrier_count(a.S, bar_target, timed_out, a.budget);
  };

  // ---- start: x = 0, r = b, the owned rows' block inverses into shared memory, u = M^-1 r, w = S u
  owned([&](int64_t k, int l) {
    sx[l] = 0;
    sr[l] = a.b[k];
    const T* M = a.Minv + (size_t)(k / 6) * BS2 + 6 * (k % 6);
#pragma unroll
    for (int j = 0; j < 6; ++j) sM[6 * (size_t)l + j] = M[j];
  });
  __syncthreads();
  double ru, rrl, wu;
  precondition(ru, rrl);
  cta_sum2<NT>(ru, rrl, cta_out);
  if (threadIdx.x == 0) { slot(0, 0)[c] = cta_out[0]; slot(0, 1)[c] = cta_out[1]; }
  double rr = 0, gam = 0, bb = 0;
  int it = 0;
  bool go = sync();
  if (go) {
    spmv(wu);
    cta_sum2<NT>(wu, 0.0, cta_out);
    if (threadIdx.x == 0) slot(0, 2)[c] = cta_out[0];
    go = sync();
  }
  auto reduce3 = [&](int par) {
    double s0 = 0, s1 = 0, s2 = 0;
    for (int g = threadIdx.x; g < G; g += NT) {
      s0 += __ldcg(&slot(par, 0)[g]);
      s1 += __ldcg(&slot(par, 1)[g]);
      s2 += __ldcg(&slot(par, 2)[g]);
    }
    s0 = warp_sum(s0);
    s1 = warp_sum(s1);
    s2 = warp_sum(s2);
    if (lane == 0) { red3[warp][0] = s0; red3[warp][1] = s1; red3[warp][2] = s2; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double t0 = 0, t1 = 0, t2 = 0;
      for (int w = 0; w < NW; ++w) { t0 += red3[w][0]; t1 += red3[w][1]; t2 += red3[w][2]; }
      bc[0] = t0; bc[1] = t1; bc[2] = t2;
    }
    __syncthreads();
  };
  bool done = !go;
  double alpha = 0, beta = 0;
  if (!done) {
    add_carries();   // ordered before the vector updates by the barriers inside reduce3
    reduce3(0);
    gam = bc[0];
    bb = bc[1];
    alpha = bc[2] > 0 ? gam / bc[2] : 0.0;
    rr = bb;
    done = !(bb > 0) || !(bc[2] > 0);
  }
  const double tol2 = a.tol * a.tol * bb;
  int par = 1;
  while (!done) {
    const bool first = it == 0;
    owned([&](int64_t, int l) {
      const double pk = first ? su[l] : su[l] + beta * sp[l];
      const double sk = first ? sw[l] : sw[l] + beta * ss[l];
      sp[l] = pk;
      ss[l] = sk;
      sx[l] += alpha * pk;
      sr[l] -= alpha * sk;
    });
    __syncthreads();
    precondition(ru, rrl);
    cta_sum2<NT>(ru, rrl, cta_out);
    if (threadIdx.x == 0) { slot(par, 0)[c] = cta_out[0]; slot(par, 1)[c] = cta_out[1]; }
    ++it;
    if (!sync()) break;
    spmv(wu);
    cta_sum2<NT>(wu, 0.0, cta_out);
    if (threadIdx.x == 0) slot(par, 2)[c] = cta_out[0];
    if (!sync()) break;
    add_carries();
    reduce3(par);
    const double gam_new = bc[0], delta = bc[2];
    rr = bc[1];
    if (rr <= tol2 || it >= a.max_iters || !(rr == rr)) break;
    beta = gam_new / gam;
    const double den = delta - beta * gam_new / alpha;
    alpha = gam_new / den;
    gam = gam_new;
    if (!(den > 0)) break;   // S not positive definite along p (rounding): keep the current x
    par ^= 1;
  }
  drain();
  __syncthreads();
  owned([&](int64_t k, int l) { a.x[k] = sx[l]; });   // the solution of the owned values
  if (timed_out) atomicOr(&a.S->flags, PCG_FLAG_TIMEOUT);
  if (c == 0 && threadIdx.x == 0) {
    a.S->iters = it;
    a.S->rr = rr;
    a.S->bnorm2 = bb;
    a.S->rz = gam;
    a.S->done = 1;
  }
}

// ============================================================================
// K7: back-substitution and the predicted decrease
// ============================================================================
template <class T>
struct BackArgs {
  const int32_t *fslot_off, *slot_ent, *slot_feat, *feat_plane_slot;
  const uint8_t* slot_type;
  const double *V, *Vinv, *g, *x;
  const T *W, *H, *G, *C;
  const T* CK;              // refined intrinsics: camera slots' blocks with their own entity (else null)
  const T* CS;              // surface groups: camera slots' blocks with the feature's sphere / cylinder / cone
  const int32_t* cam_k;     // refined intrinsics: per camera its entity (else null)
  int64_t kbase;            // A index of intrinsics entity 0
  int64_t nfp;              // features including the wireframe-coupled points' (zero-dimension, after nf)
  T* sv;        // per slot: W_e da (4, zero-padded), G_e . da, da^T H_e da + 2 da^T C_e dplane
  double* df;
  int64_t np, nf, ne;
  DevScalars* S;
  double* red;
};

// The slot part (a thread per slot, records read coalesced): the slot's share of t_f = g_f + sum_e W_e da and
// of the predicted decrease.
template <class T>
__device__ void backsub_slot(const BackArgs<T>& a, int64_t e) {
  const int64_t f = a.slot_feat[e];
  const int K = f < a.np ? 3 : 4;
  // the entity's increments in three 16-byte loads (x is 256-byte aligned, a block row 48 bytes)
  const double2* da = reinterpret_cast<const double2*>(a.x + 6 * (size_t)a.slot_ent[e]);
  T dv[6];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const double2 v = da[j];
    dv[2 * j] = (T)v.x;
    dv[2 * j + 1] = (T)v.y;
  }
  T W[24];
  if (K == 3) {   // a point's W has three rows
    load16<T, 18>(a.W + (size_t)e * SW, W);
#pragma unroll
    for (int j = 18; j < 24; ++j) W[j] = 0;
  } else {
    load16<T, 24>(a.W + (size_t)e * SW, W);
  }
  T* so = a.sv + (size_t)e * SBS;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    T s = 0;
#pragma unroll
    for (int j = 0; j < 6; ++j) s += W[i * 6 + j] * dv[j];
    so[i] = s;
  }
  T gh[SG];   // G (6), H (21), pad
  load16<T, SG>(a.G + (size_t)e * SG, gh);
  const T* G = gh;
  const T* H = gh + HG_H;
  T gd = 0, hq = 0;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    gd += G[i] * dv[i];
    T hv = 0;
#pragma unroll
    for (int j = 0; j < 6; ++j) hv += H[i <= j ? up_idx(i, j, 6) : up_idx(j, i, 6)] * dv[j];
    hq += dv[i] * hv;
  }
  T cpl = 0;
  const int pslot = a.feat_plane_slot[f];
  if (pslot >= 0 && a.slot_type[e] == ENT_CAM && ent_surface(a.slot_type[pslot])) {
    // camera-surface direct block of a feature on a sphere, cylinder, cone or 9-parameter group (6 x 6, zeros
    // beyond its dims), and a 9-parameter group's second entity (the camera slot's CK record, 6 x 3)
    const double* dp = a.x + 6 * (size_t)a.slot_ent[pslot];
    T Cm[36];
    load16<T, 36>(a.CS + (size_t)e * SCS, Cm);
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int j = 0; j < 6; ++j) cpl += dv[i] * Cm[i * 6 + j] * (T)dp[j];
    if (pslot + 1 < a.fslot_off[f + 1] && ent_second(a.slot_type[pslot + 1])) {
      const double* d2 = a.x + 6 * (size_t)a.slot_ent[pslot + 1];
      T Ck[18];
      load16<T, 18>(a.CK + (size_t)e * SC, Ck);
#pragma unroll
      for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) cpl += dv[i] * Ck[i * 3 + j] * (T)d2[j];
    }
  } else if (ent_second(a.slot_type[e])) {
    // a 9-parameter group's second entity: its coupling with the first (J_1^T w J_2, the slot's C record)
    const double* d1 = a.x + 6 * (size_t)a.slot_ent[e - 1];
    T Cm[18];
    load16<T, 18>(a.C + (size_t)e * SC, Cm);
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) cpl += (T)d1[i] * Cm[i * 3 + j] * dv[j];
  } else if (pslot >= 0 && a.slot_type[e] == ENT_CAM) {   // camera-plane direct block of a plane feature
    const double* dp = a.x + 6 * (size_t)a.slot_ent[pslot];
    const T dpl[3] = {(T)dp[0], (T)dp[1], (T)dp[2]};
    T Cm[18];
    load16<T, 18>(a.C + (size_t)e * SC, Cm);
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) cpl += dv[i] * Cm[i * 3 + j] * dpl[j];
  }
  if (f >= a.nf) {
    // a wireframe-coupled point's residuals: a camera slot's direct block with the point (the CK record, the
    // point slot is the feature's last), the point slot's with the plane (its C record, 3 x 3)
    if (a.slot_type[e] == ENT_CAM) {
      const double* dk = a.x + 6 * (size_t)a.slot_ent[a.fslot_off[f + 1] - 1];
      const T dkv[3] = {(T)dk[0], (T)dk[1], (T)dk[2]};
      T Ck[18];
      load16<T, 18>(a.CK + (size_t)e * SC, Ck);
#pragma unroll
      for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) cpl += dv[i] * Ck[i * 3 + j] * dkv[j];
    } else if (a.slot_type[e] == ENT_JPT && pslot >= 0) {
      const double* dp = a.x + 6 * (size_t)a.slot_ent[pslot];
      const T dpl[3] = {(T)dp[0], (T)dp[1], (T)dp[2]};
      T Cm[18];
      load16<T, 18>(a.C + (size_t)e * SC, Cm);
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) cpl += dv[i] * Cm[i * 3 + j] * dpl[j];
    }
  } else if (a.cam_k) {
    // refined intrinsics: a camera slot's direct block with its own entity, an intrinsics slot's with the plane
    if (a.slot_type[e] == ENT_CAM) {
      const double* dk = a.x + 6 * (size_t)(a.kbase + a.cam_k[a.slot_ent[e]]);
      const T dkv[3] = {(T)dk[0], (T)dk[1], (T)dk[2]};
      T Ck[18];
      load16<T, 18>(a.CK + (size_t)e * SC, Ck);
#pragma unroll
      for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) cpl += dv[i] * Ck[i * 3 + j] * dkv[j];
    } else if (a.slot_type[e] == ENT_INTR && pslot >= 0) {
      const double* dp = a.x + 6 * (size_t)a.slot_ent[pslot];
      const T dpl[3] = {(T)dp[0], (T)dp[1], (T)dp[2]};
      T Cm[18];
      load16<T, 18>(a.C + (size_t)e * SC, Cm);
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) cpl += dv[i] * Cm[i * 3 + j] * dpl[j];
    }
  }
  so[4] = gd;
  so[5] = hq + T(2) * cpl;
}

// The feature part: delta_f = -V^-1 t_f, and the feature's share of g.delta and delta^T H delta:
//   g_f.df + sum_e G_e.da   and   df^T V df + 2 (t_f - g_f).df + sum_e (da^T H_e da + 2 da^T C_e dplane)
// where (t_f - g_f).df = sum_e (W_e da).df is the feature-camera cross term.
template <class T, int K>
__device__ void backsub_feature(const BackArgs<T>& a, int64_t f, double& gTd, double& dHd) {
  double t[K];
  double gd = 0, hh = 0;
  if constexpr (sizeof(T) == 4) {
    // the slots' float values summed in double-single (TwoSum, as exact as an FP64 sum of them) and converted
    // once: a conversion per slot and component would cost an FP64-pipe operation on this part
    float hs[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, ls[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int e = a.fslot_off[f]; e < a.fslot_off[f + 1]; ++e) {
      const T* so = a.sv + (size_t)e * SBS;
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        if (i < K || i >= 4) two_sum_acc(hs[i], ls[i], so[i], 0.f);
      }
    }
#pragma unroll
    for (int i = 0; i < K; ++i) t[i] = a.g[4 * f + i] + ((double)hs[i] + (double)ls[i]);
    gd = (double)hs[4] + (double)ls[4];
    hh = (double)hs[5] + (double)ls[5];
  } else {
#pragma unroll
    for (int i = 0; i < K; ++i) t[i] = a.g[4 * f + i];
    for (int e = a.fslot_off[f]; e < a.fslot_off[f + 1]; ++e) {
      const T* so = a.sv + (size_t)e * SBS;
#pragma unroll
      for (int i = 0; i < K; ++i) t[i] += (double)so[i];
      gd += (double)so[4];
      hh += (double)so[5];
    }
  }
  double dfv[K];
  const double* Vi = a.Vinv + 10 * f;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    double s = 0;
#pragma unroll
    for (int j = 0; j < K; ++j) s += Vi[i <= j ? up_idx(i, j, K) : up_idx(j, i, K)] * t[j];
    dfv[i] = -s;
    a.df[4 * f + i] = -s;
  }
  const double* Vf = a.V + 10 * f;
  double vq = 0, gfd = 0, cross = 0;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    gfd += a.g[4 * f + i] * dfv[i];
    cross += (t[i] - a.g[4 * f + i]) * dfv[i];
#pragma unroll
    for (int j = 0; j < K; ++j) vq += dfv[i] * Vf[i <= j ? up_idx(i, j, K) : up_idx(j, i, K)] * dfv[j];
  }
  gTd = gfd + gd;
  dHd = vq + 2.0 * cross + hh;
}

template <class T>
__global__ void __launch_bounds__(128) k_backsub_slots(BackArgs<T> a) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < a.ne) backsub_slot<T>(a, e);
}

template <class T>
__global__ void __launch_bounds__(128) k_backsub(BackArgs<T> a) {
  int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double v[2] = {0, 0};
  if (f < a.nf) {
    if (f < a.np) backsub_feature<T, 3>(a, f, v[0], v[1]);
    else backsub_feature<T, 4>(a, f, v[0], v[1]);
  } else if (f < a.nfp) {
    // a wireframe-coupled point's residuals: their slots' shares of g.delta and delta^T H delta alone
    for (int e = a.fslot_off[f]; e < a.fslot_off[f + 1]; ++e) {
      const T* so = a.sv + (size_t)e * SBS;
      v[0] += (double)so[4];
      v[1] += (double)so[5];
    }
  }
  double tot[2];
  if (grid_reduce<2>(v, a.red, &a.S->counter[3], tot) && threadIdx.x == 0) {
    a.S->gTd = tot[0];
    a.S->dHd = tot[1];
    a.S->pred = -tot[0] - 0.5 * tot[1];
  }
}

// ============================================================================
// K8: candidate parameters (retractions) and the FP64 cost
// ============================================================================
__device__ void so3_exp(const double* w, double* R) {
  double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  double A, B;
  if (th2 < 1e-12) {
    A = 1 - th2 / 6;
    B = 0.5 - th2 / 24;
  } else {
    double th = sqrt(th2);
    A = sin(th) / th;
    B = (1 - cos(th)) / th2;
  }
  double K[9] = {0, -w[2], w[1], w[2], 0, -w[0], -w[1], w[0], 0};
  double K2[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0;
      for (int k = 0; k < 3; ++k) s += K[3 * i + k] * K[3 * k + j];
      K2[3 * i + j] = s;
    }
  for (int i = 0; i < 9; ++i) R[i] = (i % 4 == 0 ? 1.0 : 0.0) + A * K[i] + B * K2[i];
}

__device__ void s2_exp(const double* n, const double* v, double* o) {
  double th2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  double c, s;
  if (th2 < 1e-12) {
    c = 1 - th2 / 2;
    s = 1 - th2 / 6;
  } else {
    double th = sqrt(th2);
    c = cos(th);
    s = sin(th) / th;
  }
  for (int i = 0; i < 3; ++i) o[i] = c * n[i] + s * v[i];
}

struct CandArgs {
  const double *cam, *pts, *lin, *pln, *vps, *x, *df;
  const uint8_t* fixed;
  double *cam2, *pts2, *lin2, *pln2, *vps2;
  int64_t nc, np, nl, npl, nv;
  // refined intrinsics (else nk = 0): entities, their candidate values, every camera's entity, A index of entity 0
  const double* intr;
  double* intr2;
  const int32_t* cam_k;
  int64_t nk, kbase;
  // surface groups (else none): spheres, cylinders, cones (SRF_STRIDE values each), A index of the first
  const double* srf;
  double* srf2;
  int64_t nsp, ncy, nco, sbase;
  // 9-parameter groups (else none): ellipsoids then cuboids (BOX_STRIDE values each), A index of the first
  // ellipsoid's first entity
  const double* bx;
  double* bx2;
  int64_t nel, ncu, bbase;
  // 3D wireframe distance (else null): per point its index among the coupled points (-1: a feature), A index of
  // the first coupled point
  const int32_t* jq;
  int64_t jbase;
};

// the orthonormal update of a Pluecker line (d, m), |d| = 1: U <- U Exp(dl[0:3]), phi <- phi + dl[3]
__device__ void line_retract(const double* L, const double* dl, double* o);

// items: cameras, planes, VPs, points, lines, the intrinsics entities, the surface groups, then the
// 9-parameter groups
__device__ void candidate_item(const CandArgs& a, int64_t i) {
  const int64_t n0 = a.nc, n1 = n0 + a.npl, n2 = n1 + a.nv, n3 = n2 + a.np;
  if (i >= n3 + a.nl + a.nk + a.nsp + a.ncy + a.nco) {
    // ellipsoid (R <- Exp(dw) R, c + dc, s exp(ds)) or cuboid (R <- Exp(dw) R, offsets + dd): the first
    // entity's increments (dw, then dc or d_0..2), the second's (ds or d_3..5)
    const int64_t g = i - (n3 + a.nl + a.nk + a.nsp + a.ncy + a.nco);
    const bool ell = g < a.nel;
    const double* G = a.bx + BOX_STRIDE * g;
    double* o = a.bx2 + BOX_STRIDE * g;
    const int64_t e1 = ell ? a.bbase + g : a.bbase + 2 * a.nel + (g - a.nel);
    const int64_t e2 = ell ? a.bbase + a.nel + g : a.bbase + 2 * a.nel + a.ncu + (g - a.nel);
    const double* d1 = a.x + 6 * e1;
    const double* d2 = a.x + 6 * e2;
    double E[9];
    so3_exp(d1, E);
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) o[3 * r + c] = E[3 * r] * G[c] + E[3 * r + 1] * G[3 + c] + E[3 * r + 2] * G[6 + c];
    for (int k = 0; k < 3; ++k) {
      o[9 + k] = G[9 + k] + d1[3 + k];
      o[12 + k] = ell ? G[12 + k] * exp(d2[k]) : G[12 + k] + d2[k];
    }
    o[15] = G[15];
    return;
  }
  if (i >= n3 + a.nl + a.nk) {
    // sphere (c + dc, r exp(ds)), cylinder (line update of the axis, r exp(ds)), cone (a + da, axis on S^2,
    // half-angle + d)
    const int64_t g = i - n3 - a.nl - a.nk;
    const double* G = a.srf + SRF_STRIDE * g;
    double* o = a.srf2 + SRF_STRIDE * g;
    const double* dl = a.x + 6 * (a.sbase + g);
    for (int k = 0; k < SRF_STRIDE; ++k) o[k] = G[k];
    if (g < a.nsp) {
      for (int k = 0; k < 3; ++k) o[k] = G[k] + dl[k];
      o[3] = G[3] * exp(dl[3]);
    } else if (g < a.nsp + a.ncy) {
      line_retract(G, dl, o);
      o[6] = G[6] * exp(dl[4]);
    } else {
      for (int k = 0; k < 3; ++k) o[k] = G[k] + dl[k];
      double b1[3], b2[3], v[3];
      tangent_basis_d(G + 3, b1, b2);
      for (int k = 0; k < 3; ++k) v[k] = dl[3] * b1[k] + dl[4] * b2[k];
      s2_exp(G + 3, v, o + 3);
      o[6] = G[6] + dl[5];
    }
    return;
  }
  if (i >= n3 + a.nl) {
    // intrinsics entity: additive (f, k1, k2)
    const int64_t k = i - n3 - a.nl;
    for (int j = 0; j < 3; ++j) a.intr2[3 * k + j] = a.intr[3 * k + j] + a.x[6 * (a.kbase + k) + j];
    return;
  }
  if (i < n0) {
    const double* c = a.cam + 12 * i;
    double* o = a.cam2 + 12 * i;
    for (int k = 0; k < 12; ++k) o[k] = c[k];
    if (a.nk) {
      // the camera's f, k1, k2: its entity's candidate values (the same sums as the entity's item)
      const int64_t k = a.cam_k[i];
      for (int j = 0; j < 3; ++j) o[7 + j] = a.intr[3 * k + j] + a.x[6 * (a.kbase + k) + j];
    }
    if (a.fixed[i] == 0x3F) return;
    const double* dl = a.x + 6 * i;   // held components have zero increments
    double Rd[9], R[9], Rn[9];
    so3_exp(dl, Rd);
    quat_to_R(c, R);
    for (int r = 0; r < 3; ++r)
      for (int s = 0; s < 3; ++s) Rn[3 * r + s] = Rd[3 * r] * R[s] + Rd[3 * r + 1] * R[3 + s] + Rd[3 * r + 2] * R[6 + s];
    // rotation matrix -> quaternion (w >= 0)
    double q[4];
    double tr = Rn[0] + Rn[4] + Rn[8];
    if (tr > 0) {
      double s = sqrt(tr + 1.0) * 2;
      q[0] = 0.25 * s; q[1] = (Rn[7] - Rn[5]) / s; q[2] = (Rn[2] - Rn[6]) / s; q[3] = (Rn[3] - Rn[1]) / s;
    } else if (Rn[0] > Rn[4] && Rn[0] > Rn[8]) {
      double s = sqrt(1.0 + Rn[0] - Rn[4] - Rn[8]) * 2;
      q[0] = (Rn[7] - Rn[5]) / s; q[1] = 0.25 * s; q[2] = (Rn[1] + Rn[3]) / s; q[3] = (Rn[2] + Rn[6]) / s;
    } else if (Rn[4] > Rn[8]) {
      double s = sqrt(1.0 + Rn[4] - Rn[0] - Rn[8]) * 2;
      q[0] = (Rn[2] - Rn[6]) / s; q[1] = (Rn[1] + Rn[3]) / s; q[2] = 0.25 * s; q[3] = (Rn[5] + Rn[7]) / s;
    } else {
      double s = sqrt(1.0 + Rn[8] - Rn[0] - Rn[4]) * 2;
      q[0] = (Rn[3] - Rn[1]) / s; q[1] = (Rn[2] + Rn[6]) / s; q[2] = (Rn[5] + Rn[7]) / s; q[3] = 0.25 * s;
    }
    double sg = q[0] < 0 ? -1.0 : 1.0;
    double qn = sg / sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int k = 0; k < 4; ++k) o[k] = q[k] * qn;
    o[4] = c[4] + dl[3]; o[5] = c[5] + dl[4]; o[6] = c[6] + dl[5];
  } else if (i < n1) {
    int64_t g = i - n0;
    const double* P = a.pln + 4 * g;
    const double* dl = a.x + 6 * i;
    double b1[3], b2[3], v[3];
    tangent_basis_d(P, b1, b2);
    for (int k = 0; k < 3; ++k) v[k] = dl[0] * b1[k] + dl[1] * b2[k];
    double* o = a.pln2 + 4 * g;
    s2_exp(P, v, o);
    o[3] = P[3] + dl[2];
  } else if (i < n2) {
    int64_t g = i - n1;
    const double* V = a.vps + 3 * g;
    const double* dl = a.x + 6 * i;
    double b1[3], b2[3], v[3];
    tangent_basis_d(V, b1, b2);
    for (int k = 0; k < 3; ++k) v[k] = dl[0] * b1[k] + dl[1] * b2[k];
    s2_exp(V, v, a.vps2 + 3 * g);
  } else if (i < n3) {
    int64_t f = i - n2;
    const double* dl = (a.jq && a.jq[f] >= 0) ? a.x + 6 * (a.jbase + a.jq[f]) : a.df + 4 * f;
    for (int k = 0; k < 3; ++k) a.pts2[3 * f + k] = a.pts[3 * f + k] + dl[k];
  } else {
    const int64_t l = i - n3;
    line_retract(a.lin + 6 * l, a.df + 4 * (a.np + l), a.lin2 + 6 * l);
  }
}

__device__ void line_retract(const double* L, const double* dl, double* o) {
  double u1[3], u3[3], r;
  line_frame<double>(L, L + 3, u1, u3, r);
  double E[9];
  so3_exp(dl, E);
  // U = [u1, d, u3] (columns); U' = U E
  double U[9] = {u1[0], L[0], u3[0], u1[1], L[1], u3[1], u1[2], L[2], u3[2]};
  double Un[9];
  for (int rr = 0; rr < 3; ++rr)
    for (int s = 0; s < 3; ++s) Un[3 * rr + s] = U[3 * rr] * E[s] + U[3 * rr + 1] * E[3 + s] + U[3 * rr + 2] * E[6 + s];
  double phi = atan2(1.0, r) + dl[3];
  double ct = cos(phi) / sin(phi);
  double d[3], m[3];   // computed in full before writing: o may alias nothing the caller still reads
  for (int k = 0; k < 3; ++k) {
    d[k] = Un[3 * k + 1];
    m[k] = ct * Un[3 * k + 0];
  }
  for (int k = 0; k < 3; ++k) { o[k] = d[k]; o[3 + k] = m[k]; }
}

__global__ void k_candidate(CandArgs a) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < a.nc + a.npl + a.nv + a.np + a.nl + a.nk + a.nsp + a.ncy + a.nco + a.nel + a.ncu) candidate_item(a, i);
}

// ---- ln(1 + x) for the FP64 cost, table-driven after P. T. P. Tang, "Table-driven implementation of the
// logarithm function in IEEE floating-point arithmetic", ACM TOMS 16(4), 1990, with D. Goldberg's correction
// for the rounding of 1 + x.  With u = 1 + x = 2^k m, m in [1, 2), and c_j = 1 + j/64 the left end of m's
// 1/64 interval: ln u = k ln 2 - ln(rc_j) + ln(1 + d), d = m rc_j - 1 in [0, 2^-6) (rc_j = 1/c_j rounded, and
// the table holds -ln(rc_j) so that the rounding of rc_j cancels exactly), ln(1 + d) by its Taylor series to
// degree 9 (remainder below 2^-60 relative).  Every term is non-negative, and for j = 0 the table entries are
// exactly 1 and 0, so nothing cancels as x -> 0.
__device__ double g_ln1p_tab[130];   // j < 64: rc_j, -ln(rc_j); then ln 2 split into a 28-bit head and a tail

__global__ void k_ln1p_table() {
  const int j = threadIdx.x;
  if (j < 64) {
    const double rc = 1.0 / (1.0 + j / 64.0);
    g_ln1p_tab[2 * j] = rc;
    g_ln1p_tab[2 * j + 1] = -log(rc);
  } else if (j == 64) {
    const double l2 = log(2.0);
    const double hi = __longlong_as_double(__double_as_longlong(l2) & ~0xffffffLL);   // k * hi is exact
    g_ln1p_tab[128] = hi;
    g_ln1p_tab[129] = l2 - hi;
  }
}

__device__ __forceinline__ double ln1p_tab(double x) {
  const double u = 1.0 + x;
  if (!(u >= 1.0 && u <= 1.0e308)) return log1p(x);   // negative arguments, infinity and NaN
  const double corr = (x - (u - 1.0)) * (double)__frcp_rn((float)u);   // the rounding error of 1 + x, over u
  const long long b = __double_as_longlong(u);
  const int k = (int)(b >> 52) - 1023;
  const int j = (int)((b >> 46) & 63);
  const double m = __longlong_as_double((b & 0x000fffffffffffffLL) | 0x3ff0000000000000LL);
  const double d = fma(m, __ldg(&g_ln1p_tab[2 * j]), -1.0);
  double p = 1.0 / 9;
  p = fma(p, d, -1.0 / 8);
  p = fma(p, d, 1.0 / 7);
  p = fma(p, d, -1.0 / 6);
  p = fma(p, d, 1.0 / 5);
  p = fma(p, d, -1.0 / 4);
  p = fma(p, d, 1.0 / 3);
  p = fma(p, d, -1.0 / 2);
  p = fma(p, d, 1.0);
  const double kd = (double)k;
  return fma(kd, __ldg(&g_ln1p_tab[128]), __ldg(&g_ln1p_tab[2 * j + 1]) + fma(kd, __ldg(&g_ln1p_tab[129]), fma(p, d, corr)));
}

// fills the table once per device (stream-ordered, then synchronised so that every stream sees it)
cudaError_t ensure_ln1p_table(cudaStream_t st) {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> g(mu);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (done[dev]) return cudaSuccess;
  k_ln1p_table<<<1, 96, 0, st>>>();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  done[dev] = true;
  return cudaSuccess;
}

// ln(1 + x) of n device values exactly as the cost pass evaluates it (inspection of the logarithm)
__global__ void k_ln1p_eval(int64_t n, const double* __restrict__ x, double* __restrict__ y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = ln1p_tab(x[i]);
}

cudaError_t launch_ln1p_eval(cudaStream_t st, int64_t n, const double* x, double* y) {
  cudaError_t e = ensure_ln1p_table(st);
  if (e != cudaSuccess || n <= 0) return e;
  k_ln1p_eval<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, x, y);
  return cudaGetLastError();
}

struct CostArgs {
  const int8_t* rkind;
  const int32_t *rcam, *rfeat, *rgrp, *order;
  const int32_t* partner;   // per point record its plane-induced partner (or -1), or null: every record alone
  const double *meas, *camD, *grpD, *pts, *lin;
  const double* srf;   // surface groups (spheres, cylinders, cones)
  const double* bx;    // 9-parameter groups (ellipsoids, cuboids)
  int64_t nr, np, npl, nsp, ncy, nel;
  LossW loss;
  DevScalars* S;
  double* red;
  int candidate;
};

// EXT: the sphere ... cuboid kinds too (a separate instantiation, so that the common kinds' kernel keeps its
// registers and code size)
// the Cauchy term of one residual's squared norm s (its share of E and of E_px)
__device__ __forceinline__ void cost_term(const CostArgs& a, int kind, double s, double (&v)[2]) {
  const double e = a.loss.half_wa2[kind] * ln1p_tab(s * a.loss.inv_a2[kind]);
  v[0] += e;
  if (res_pixel(kind)) v[1] += e;
}

// a point record and its plane-induced partner (Eq. 1 and Eq. 7 for the same point and camera): pi(C, X)
// once, each residual formed with the operations of res_point and res_plane_point
__device__ void cost_point_pair(const CostArgs& a, int64_t i, int64_t j, double (&v)[2]) {
  const int cid = a.rcam[i];
  const double* X = a.pts + 3 * (size_t)a.rfeat[i];
  const double* meas = a.meas + 4 * i;
  const double* P = a.grpD + (size_t)GRP_STRIDE * a.rgrp[j];
  Cam<double> c;
  load_cam(a.camD + (size_t)CAM_STRIDE * cid, c);
  double p1[3], x1[3], pi1[2], J1[2][3];
  matvec3(c.R, X, p1);
#pragma unroll
  for (int k = 0; k < 3; ++k) x1[k] = p1[k] + c.t[k];
  if (!(x1[2] > 1e-6)) return;   // both residuals invalid
  project_dist<double, false>(c, x1, pi1, J1);
  const double r0 = pi1[0] - meas[0], r1 = pi1[1] - meas[1];
  cost_term(a, R_POINT, r0 * r0 + r1 * r1, v);
  double Xp[3], cd, p2[3], x2[3], pi2[2], J2[2][3];
  plane_proj_point(P, P[3], X, Xp, cd);
  matvec3(c.R, Xp, p2);
#pragma unroll
  for (int k = 0; k < 3; ++k) x2[k] = p2[k] + c.t[k];
  if (!(x2[2] > 1e-6)) return;
  project_dist<double, false>(c, x2, pi2, J2);
  const double q0 = pi1[0] - pi2[0], q1 = pi1[1] - pi2[1];
  cost_term(a, R_PLANE_POINT, q0 * q0 + q1 * q1, v);
}

template <bool EXT = false>
__device__ void cost_residual(const CostArgs& a, int64_t i, double (&v)[2]) {
  if (a.partner && a.rkind[i] == R_POINT) {
    const int32_t j = a.partner[i];
    if (j >= 0) {
      cost_point_pair(a, i, j, v);
      return;
    }
  }
  {
    const int kind = a.rkind[i];
    const int cid = a.rcam[i];
    const int64_t f = a.rfeat[i];
    const int gid = a.rgrp[i];
    const double* meas = a.meas + 4 * i;
    Cam<double> c;
    if (cid >= 0) load_cam(a.camD + (size_t)CAM_STRIDE * cid, c);
    ResJ<double> o;
    o.valid = false;
    const double* X = a.pts + 3 * f;
    const double* L = a.lin + 6 * (f - a.np);
    int rd = res_dim(kind);
    switch (kind) {
      case R_POINT: res_point<double, false>(c, X, meas, o); break;
      case R_LINE: res_line<double, false>(c, L, meas, o); break;
      case R_PLANE_POINT: res_plane_point<double, false>(c, X, a.grpD + (size_t)GRP_STRIDE * gid, o); break;
      case R_PLANE_LINE: res_plane_line<double, false>(c, L, a.grpD + (size_t)GRP_STRIDE * gid, meas, o); break;
      case R_VP: res_vp<double, false>(L, a.grpD + (size_t)GRP_STRIDE * (a.npl + gid), o); break;
      case R_P2L: res_p2l<double, false>(c, X, meas, o); break;
      case R_L2P: res_l2p<double, false>(c, L, meas, o); break;
      case R_PLANE_POINT3: res_plane_point3<double, false>(X, a.grpD + (size_t)GRP_STRIDE * gid, o); break;
      case R_PLANE_LINE3: res_plane_line3<double, false>(L, a.grpD + (size_t)GRP_STRIDE * gid, o); break;
      default:
        if constexpr (EXT) {
          switch (kind) {
            case R_SPHERE_POINT: res_surface_point<double, false, 0>(c, X, a.srf + (size_t)SRF_STRIDE * gid, o); break;
            case R_CYL_POINT: res_surface_point<double, false, 1>(c, X, a.srf + (size_t)SRF_STRIDE * (a.nsp + gid), o); break;
            case R_CONE_POINT: res_surface_point<double, false, 2>(c, X, a.srf + (size_t)SRF_STRIDE * (a.nsp + a.ncy + gid), o); break;
            case R_ELL_POINT: res_box_point<double, false, 3>(c, X, a.bx + (size_t)BOX_STRIDE * gid, o); break;
            case R_CUB_POINT: res_box_point<double, false, 4>(c, X, a.bx + (size_t)BOX_STRIDE * (a.nel + gid), o); break;
            case R_WF3D: res_wf3d<double, false>(L, a.pts + 3 * (size_t)gid, o); break;
            case R_CUB_LINE: res_box_line<double, false>(c, L, a.bx + (size_t)BOX_STRIDE * (a.nel + gid), meas, o); break;
          }
        }
        break;
    }
    if (o.valid) {
      double s = 0;
      for (int k = 0; k < rd; ++k) s += o.r[k] * o.r[k];
      cost_term(a, kind, s, v);
    }
  }
}

// a grid of a few CTAs per SM striding over the residuals: the FP64 pipe bounds this pass, and the SMs keep
// room for the candidate's linearisation that runs beside it on another stream
template <bool EXT>
__global__ void __launch_bounds__(256) k_cost(CostArgs a) {
  double v[2] = {0, 0};
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < a.nr; t += (int64_t)gridDim.x * blockDim.x) {
    double w[2] = {0, 0};
    cost_residual<EXT>(a, a.order[t], w);
    v[0] += w[0];
    v[1] += w[1];
  }
  double tot[2];
  if (grid_reduce<2>(v, a.red, &a.S->counter[4], tot) && threadIdx.x == 0) {
    if (a.candidate) { a.S->Enew = tot[0]; a.S->Epxnew = tot[1]; }
    else { a.S->E = tot[0]; a.S->Epx = tot[1]; }
  }
}

// ============================================================================
// K9: LM decision
// ============================================================================
struct DecideArgs {
  DevScalars* S;
  double min_gain, lmin, lmax;
};

__device__ void decide(const DecideArgs& a) {
  DevScalars* S = a.S;
  double pred = S->pred;
  double gain = pred > 0 ? (S->E - S->Enew) / pred : -INFINITY;
  bool ok = isfinite(S->Enew) && gain > a.min_gain;
  S->gain = gain;
  S->accepted = ok ? 1 : 0;
  if (ok) {
    double t = 2.0 * gain - 1.0;
    double fct = fmax(1.0 / 3.0, 1.0 - t * t * t);
    S->lambda = fmin(fmax(S->lambda * fct, a.lmin), a.lmax);
    S->nu = 2.0;
  } else {
    S->lambda = fmin(S->lambda * S->nu, a.lmax);
    S->nu *= 2.0;
  }
}

__global__ void k_decide(DecideArgs a) { decide(a); }

// ============================================================================
// FMA throughput probe: the denominators of the ALU rooflines (FP32 and FP64 pipes).  Every thread runs
// eight independent FMA chains, so the pipes, not the chains' latency, bound the rate.
// ============================================================================
template <class T>
__global__ void __launch_bounds__(256) k_fma_probe(int iters, T seed, T* sink) {
  T a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = seed + (T)(threadIdx.x + k);
  const T m = (T)0.999999, c = (T)1e-7;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fma(a[k], m, c);
  T t = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) t += a[k];
  if (t == (T)-1) sink[threadIdx.x] = t;   // never true: keeps the chains live
}

cudaError_t fma_probe(int precision, double* tflops, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) || (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))) return e;
  const bool f64 = precision == BA_FP64;
  const int iters = f64 ? 1 << 12 : 1 << 16;
  const int grid = sms * 8, nt = 256;
  void* sink = nullptr;
  if ((e = cudaMalloc(&sink, 256 * sizeof(double)))) return e;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {   // the first launch warms the clocks up; the best of the rest counts
    cudaEventRecord(e0, st);
    if (f64) k_fma_probe<double><<<grid, nt, 0, st>>>(iters, 1.0, (double*)sink);
    else k_fma_probe<float><<<grid, nt, 0, st>>>(iters, 1.0f, (float*)sink);
    cudaEventRecord(e1, st);
    if ((e = cudaEventSynchronize(e1))) break;
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0) best = fminf(best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (e == cudaSuccess) e = cudaGetLastError();
  *tflops = 2.0 * 8.0 * iters * (double)grid * nt / (best * 1e-3) / 1e12;
  return e;
}

// ============================================================================
// launchers
// ============================================================================
static inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t); }

static LossW make_loss(const ba_options& o) {
  LossW L;
  // per kind: points, lines, plane-induced (2), VP, wireframe (2), direct 3D plane distances (2), sphere /
  // cylinder / cone / ellipsoid / cuboid-induced (5), the 3D wireframe endpoint distance, lines on cuboids
  const double w[N_KINDS] = {o.w_point, o.w_line, o.w_group, o.w_group, o.w_vp, o.w_wire, o.w_wire,
                             o.w_group3d, o.w_group3d, o.w_group, o.w_group, o.w_group, o.w_group, o.w_group,
                             o.w_wire3d, o.w_group};
  static_assert(N_KINDS == 16, "a weight per residual kind");
  for (int k = 0; k < N_KINDS; ++k) {
    L.w[k] = w[k];
    double s = (k == R_VP) ? o.cauchy_vp : (res_has_cam(k) ? o.cauchy_px : o.cauchy_3d);
    L.a2[k] = s * s;
    L.inv_a2[k] = 1.0 / L.a2[k];
    L.half_wa2[k] = 0.5 * w[k] * L.a2[k];
    L.wf[k] = (float)L.w[k];
    L.inv_a2f[k] = (float)L.inv_a2[k];
  }
  return L;
}


template <class T>
void launch_prepare(Problem& P, bool candidate_only, bool working_only) {
  const Dims& d = P.d;
  auto& cs = P.ps[candidate_only ? 1 - P.cur : P.cur];
  T* camW = candidate_only ? nullptr : (T*)P.camT;
  T* grpW = candidate_only ? nullptr : (T*)P.grpT;
  if (sizeof(T) == sizeof(double)) { camW = nullptr; grpW = nullptr; }
  // working_only: the float working copies alone (the derived FP64 data of this set exist already and may be
  // read by a kernel of another stream meanwhile)
  double* camD = working_only ? nullptr : cs.camD;
  double* grpD = working_only ? nullptr : cs.grpD;
  if (working_only && !camW) return;
  if (d.nc) { ++P.launches; k_derive_cams<T><<<nblk(d.nc, 128), 128, 0, P.stream>>>(d.nc, cs.cam, camD, camW); }
  if (d.npl + d.nv) { ++P.launches; k_derive_groups<T><<<nblk(d.npl + d.nv, 128), 128, 0, P.stream>>>(d.npl, d.nv, cs.pln, cs.vps, grpD, grpW); }
  if (!candidate_only && sizeof(T) == sizeof(float)) {
    if (d.ngs()) {
      ++P.launches;
      k_convert<<<nblk(SRF_STRIDE * d.ngs(), 256), 256, 0, P.stream>>>(SRF_STRIDE * d.ngs(), cs.srf, (float*)P.srfT);
    }
    if (d.nbx()) {
      ++P.launches;
      k_convert<<<nblk(BOX_STRIDE * d.nbx(), 256), 256, 0, P.stream>>>(BOX_STRIDE * d.nbx(), cs.bx, (float*)P.bxT);
    }
    if (d.np) { ++P.launches; k_convert<<<nblk(3 * d.np, 256), 256, 0, P.stream>>>(3 * d.np, cs.pts, (float*)P.ptsT); }
    if (d.nl) { ++P.launches; k_convert<<<nblk(6 * d.nl, 256), 256, 0, P.stream>>>(6 * d.nl, cs.lin, (float*)P.linT); }
  }
}

template <class T>
void launch_linearize(Problem& P) {
  const Dims& d = P.d;
  auto& cs = P.ps[P.cur];
  LinArgs<T> a;
  a.rkind = P.rkind; a.cam_mask = P.cam_fixed; a.rcam = P.rcam; a.rgrp = P.rgrp; a.rslot_c = P.rslot_c; a.rslot_g = P.rslot_g;
  a.fres_off = P.fres_off; a.feat_plane_slot = P.feat_plane_slot;
  const bool dbl = sizeof(T) == sizeof(double);
  a.meas = dbl ? (const T*)P.meas64 : (const T*)P.measT;
  a.cam = dbl ? (const T*)cs.camD : (const T*)P.camT;
  a.grp = dbl ? (const T*)cs.grpD : (const T*)P.grpT;
  a.pts = dbl ? (const T*)cs.pts : (const T*)P.ptsT;
  a.lin = dbl ? (const T*)cs.lin : (const T*)P.linT;
  a.npl = d.npl; a.np = d.np;
  a.W = (T*)P.slotW; a.H = (T*)P.slotH; a.G = (T*)P.slotG; a.C = (T*)P.slotC;
  a.V = P.featV; a.g = P.featg;
  a.loss = make_loss(P.opt);
  a.rslot_k = P.rslot_k; a.fslot_off = P.fslot_off; a.slot_type = P.slot_type; a.CK = (T*)P.slotCK;
  a.srf = dbl ? (const T*)cs.srf : (const T*)P.srfT; a.CS = (T*)P.slotCS; a.nsp = d.nsp; a.ncy = d.ncy;
  a.bx = dbl ? (const T*)cs.bx : (const T*)P.bxT; a.nel = d.nel;
  a.jp_pt = P.jp_pt; a.nf = d.nf;
  if (d.njp) {
    // 3D wireframe distances: the lines' coupled-point slots, then the coupled points' own residuals
    // (refined intrinsics and the other group types are refused together with them)
    if (d.np) { ++P.launches; k_linearize<T, 3><<<nblk(d.np, 128), 128, 0, P.stream>>>(a, 0, d.np); }
    if (d.nl) { ++P.launches; k_linearize<T, 4, false, false, true><<<nblk(d.nl, 128), 128, 0, P.stream>>>(a, d.np, d.nf); }
    ++P.launches;
    k_linearize_jpoint<T><<<nblk(d.njp, 128), 128, 0, P.stream>>>(a, d.njp);
    return;
  }
  if (d.ngs() || d.nbx()) {
    // spheres, cylinders, cones: the points' positional groups take up to 6 dimensions (refined intrinsics are
    // refused together with them)
    if (d.np) { ++P.launches; k_linearize<T, 3, false, true><<<nblk(d.np, 128), 128, 0, P.stream>>>(a, 0, d.np); }
    if (d.nl) {
      ++P.launches;
      // lines on cuboids take the 6-wide group accumulators and the cuboid's second entity too
      if (d.ncu) k_linearize<T, 4, false, true><<<nblk(d.nl, 128), 128, 0, P.stream>>>(a, d.np, d.nf);
      else k_linearize<T, 4><<<nblk(d.nl, 128), 128, 0, P.stream>>>(a, d.np, d.nf);
    }
    return;
  }
  if (d.nk) {
    // refined intrinsics: the feature's intrinsics slots and the camera slots' couplings with them too
    if (d.np) { ++P.launches; k_linearize<T, 3, true><<<nblk(d.np, 128), 128, 0, P.stream>>>(a, 0, d.np); }
    if (d.nl) { ++P.launches; k_linearize<T, 4, true><<<nblk(d.nl, 128), 128, 0, P.stream>>>(a, d.np, d.nf); }
    return;
  }
  // a warp per CTA: at 217 registers a thread, an SM holds 9 warps of one-warp CTAs against 8 of 128-thread ones
  if (d.np) { ++P.launches; k_linearize<T, 3><<<nblk(d.np, 32), 32, 0, P.stream>>>(a, 0, d.np); }
  if (d.nl) { ++P.launches; k_linearize<T, 4><<<nblk(d.nl, 128), 128, 0, P.stream>>>(a, d.np, d.nf); }
}

template <class T>
void launch_invert(Problem& P, double lambda) {
  const Dims& d = P.d;
  InvArgs<T> a;
  a.fslot_off = P.fslot_off; a.slot_feat = P.slot_feat; a.V = P.featV; a.g = P.featg; a.W = (const T*)P.slotW;
  a.G = (const T*)P.slotG; a.Vinv = P.featVinv; a.u = P.featu; a.L = P.featL; a.Z = (T*)P.slotZ; a.B = (T*)P.slotB;
  a.np = d.np; a.nf = d.nf; a.ne = d.ne; a.lambda = lambda; a.S = P.S;
  if (d.nf) { ++P.launches; k_invert<T><<<nblk(d.nf, 128), 128, 0, P.stream>>>(a); }
  if (d.ne) { ++P.launches; k_whiten<T><<<nblk(d.ne, 128), 128, 0, P.stream>>>(a); }
}

template <class T>
UnitArgs<T> unit_args(Problem& P, double lambda) {
  const Dims& d = P.d;
  BlockArgs<T> b;
  b.up_row = P.up_row; b.up_full = P.up_full; b.up_mirror = P.up_mirror; b.col = P.col;
  b.ent_type = P.ent_type; b.cam_fixed = P.cam_fixed; b.Sval = (T*)P.Sval; b.sv = sview_of(P);
  b.b = P.bvec; b.Dg = P.Dg; b.sdiag = P.sdiag; b.nc = d.nc; b.ngend = d.nc + d.npl + d.nv; b.lambda = lambda;
  b.relH = P.nrel ? P.relH : nullptr; b.relG = P.nrel ? P.relG : nullptr;
  UnitArgs<T> un;
  un.un_se = P.un_se; un.un_blk = P.un_blk; un.un_order = P.un_order; un.up_un = P.up_un; un.multi = P.multi_blk;
  un.un_desc = reinterpret_cast<const int4*>(P.un_desc); un.un_mflag = P.un_mflag;
  un.pair_a = P.pair_a; un.pair_b = P.pair_b; un.Z = (const T*)P.slotZ; un.H = (const T*)P.slotH;
  un.B = (const T*)P.slotB; un.C = (const T*)P.slotC; un.CK = (const T*)P.slotCK; un.CS = (const T*)P.slotCS;
  un.upart = P.upart;
  un.nun = d.nun; un.nmulti = d.nmulti;
  un.pk_desc = reinterpret_cast<const int4*>(P.pk_desc); un.nun_main = d.nun_main; un.npack = d.npack;
  un.line_slot0 = P.line_slot0; un.fb = b; un.ctr = P.unit_ctr;
  return un;
}

template <class T>
void launch_schur(Problem& P, double lambda) {
  const Dims& d = P.d;
  const UnitArgs<T> un = unit_args<T>(P, lambda);
  constexpr int NW = UnitWarps<T>::n;
  if (d.nun_main) {
    ++P.launches;
    cudaMemsetAsync(P.unit_ctr, 0, sizeof(int), P.stream);
    k_schur_units<T><<<schur_units_grid<T>(P.device, d.nun_main), NW * 32, (size_t)NW * UnitPipeSmem<T>::bytes,
                       P.stream>>>(un);
  }
  if (d.npack) {
    ++P.launches;
    k_schur_packs<T><<<nblk(d.npack, NW), NW * 32, 0, P.stream>>>(un);
  }
  if (P.ev[3]) cudaEventRecord(P.ev[3], P.stream);
  if (d.nmulti) { ++P.launches; k_schur_finish<T><<<nblk(d.nmulti, 128), 128, 0, P.stream>>>(un); }
}

template <class T>
void launch_precond(Problem& P) {
  const Dims& d = P.d;
  if (d.na) {
    ++P.launches;
    k_precond<T, true><<<nblk(d.na, 128), 128, 0, P.stream>>>(d.na, P.row_ptr, P.col, (const T*)P.Sval, (T*)P.Minv,
                                                              P.S, sview_of(P));
  }
}

constexpr int PCG_THREADS = 512;

// occupancy and shared-memory opt-in of the streaming PCG for `smem` bytes of chunk sums (the stage
// buffers come on top)
template <class T>
int pcg_blocks_per_sm(size_t smem) {
  constexpr int NT = StreamCfg<T>::NT, NB = StreamCfg<T>::NBUF;
  const size_t tot = smem + stream_stage_bytes<T>();
  cudaFuncSetAttribute(k_pcg_stream<T, NT, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tot);
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pcg_stream<T, NT, NB>, NT, tot);
  return nb;
}

template <class T>
void pcg_allow_smem(size_t smem) {
  constexpr int NT = StreamCfg<T>::NT, NB = StreamCfg<T>::NBUF;
  cudaFuncSetAttribute(k_pcg_stream<T, NT, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)(smem + stream_stage_bytes<T>()));
}

// the typed-storage PCG: its fixed shared memory, occupancy (with the opt-in for `smem` bytes in all)
template <class T>
size_t pcg_typed_fixed_smem(int gv) { return typed_fixed_smem<T>(gv); }

template <class T>
size_t pcg_typed_gacc_bytes(int gv) { return (size_t)(TypedCfg<T>::NT / 32) * typed_gvp<T>(gv) * sizeof(DotAcc<T>); }

template <class T>
int pcg_typed_blocks_per_sm(size_t smem) {
  constexpr int NT = TypedCfg<T>::NT, NB = TypedCfg<T>::NBUF;
  cudaFuncSetAttribute(k_pcg_typed<T, NT, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pcg_typed<T, NT, NB>, NT, smem);
  return nb;
}

template <class T>
static void launch_pcg_typed(Problem& P) {
  const Dims& d = P.d;
  constexpr int NT = TypedCfg<T>::NT, NB = TypedCfg<T>::NBUF;
  PcgTypedArgs<T> a;
  a.na = d.na; a.nc = d.nc; a.npl = d.npl; a.nv = d.nv; a.gv = P.gv;
  a.tcol = P.tcol; a.row_chunk0 = P.row_chunk0; a.gg_ptr = P.gg_ptr; a.gg_col = P.gg_col; a.cta_gs = P.cta_gs;
  a.gv_idx = P.gv_idx; a.tchunk = P.tchunk; a.cta_part = reinterpret_cast<const int4*>(P.cta_part);
  a.carry = P.pcg_carry; a.part_g = P.part_g;
  a.Sv = (const T*)P.Sval; a.Minv = (const T*)P.Minv; a.gg_val0 = P.gg_val0; a.b = P.bvec;
  a.x = P.x; a.r = P.r; a.u = P.z; a.p = P.p; a.w = P.Ap; a.s = P.svec; a.part = P.red; a.S = P.S;
  a.uhl = sizeof(T) == sizeof(float) ? P.phl : nullptr;
  a.tol = P.opt.pcg_rel_tol; a.max_iters = P.opt.pcg_max_iters;
  a.keep_frac = P.pcg_keep_frac;
  a.budget = P.opt.wait_budget_cycles > 0 ? P.opt.wait_budget_cycles : 1;
  a.nown = P.pcg_nown;
  void* args[] = {&a};
  ++P.launches;
  // the grid barriers' arrival counter starts at zero in every launch
  P.pcg_err = cudaMemsetAsync(&P.S->bar_arrive, 0, sizeof(unsigned long long), P.stream);
  if (P.pcg_err != cudaSuccess) return;
  P.pcg_err = cudaLaunchCooperativeKernel((const void*)k_pcg_typed<T, NT, NB>, dim3(P.pcg_grid), dim3(NT), args,
                                          P.pcg_smem, P.stream);
}

template <class T>
void launch_pcg(Problem& P) {
  if (P.typed) {
    launch_pcg_typed<T>(P);
    return;
  }
  const Dims& d = P.d;
  constexpr int NT = StreamCfg<T>::NT, NB = StreamCfg<T>::NBUF;
  PcgStreamArgs<T> a;
  a.na = d.na; a.col = P.col; a.row_chunk0 = P.row_chunk0; a.chunk_beg = P.chunk_beg;
  a.cta_part = reinterpret_cast<const int4*>(P.cta_part); a.carry = P.pcg_carry;
  a.Sval = (const T*)P.Sval; a.Minv = (const T*)P.Minv; a.b = P.bvec;
  a.x = P.x; a.r = P.r; a.u = P.z; a.p = P.p; a.w = P.Ap; a.s = P.svec; a.part = P.red; a.S = P.S;
  a.uhl = sizeof(T) == sizeof(float) ? P.phl : nullptr;
  a.tol = P.opt.pcg_rel_tol; a.max_iters = P.opt.pcg_max_iters;
  a.keep_frac = P.pcg_keep_frac;
  a.budget = P.opt.wait_budget_cycles > 0 ? P.opt.wait_budget_cycles : 1;
  void* args[] = {&a};
  ++P.launches;
  // the grid barriers' arrival counter starts at zero in every launch
  P.pcg_err = cudaMemsetAsync(&P.S->bar_arrive, 0, sizeof(unsigned long long), P.stream);
  if (P.pcg_err != cudaSuccess) return;
  P.pcg_err = cudaLaunchCooperativeKernel((const void*)k_pcg_stream<T, NT, NB>, dim3(P.pcg_grid), dim3(NT), args,
                                          P.pcg_smem + stream_stage_bytes<T>(), P.stream);
}

// ---- launchers on caller-provided pointers (FP64), used by the allocation-free PCG entry point
cudaError_t launch_precond_raw_f64(cudaStream_t st, int64_t na, const int32_t* row_ptr, const int32_t* col,
                                   const double* Sval, double* Minv, DevScalars* S) {
  if (na > 0) k_precond<double, false><<<nblk(na, 128), 128, 0, st>>>(na, row_ptr, col, Sval, Minv, S, SView());
  return cudaGetLastError();
}

int pcg_occupancy_f64(size_t smem) {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pcg_persistent<double, PCG_THREADS, false>, PCG_THREADS, smem);
  return nb;
}

cudaError_t launch_pcg_raw_f64(cudaStream_t st, int grid, size_t smem, int64_t na, const int32_t* col,
                               const int32_t* cta_row0, const int32_t* row_chunk0, const int32_t* chunk_beg,
                               const double* Sval, const double* Minv, const double* b, double* x, double* r,
                               double* z, double* p, double* Ap, double* part, DevScalars* S, double tol,
                               int max_iters) {
  PcgArgs<double> a;
  a.na = na; a.col = col; a.cta_row0 = cta_row0; a.row_chunk0 = row_chunk0; a.chunk_beg = chunk_beg;
  a.Sval = Sval; a.Minv = Minv; a.b = b; a.x = x; a.r = r; a.z = z; a.p = p; a.Ap = Ap; a.part = part; a.S = S;
  a.phl = nullptr;
  a.tol = tol; a.max_iters = max_iters;
  a.budget = 2000000000LL;   // about a second at the SM clock; the caller's scalars start at zero
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel((const void*)k_pcg_persistent<double, PCG_THREADS, false>, dim3(grid),
                                     dim3(PCG_THREADS), args, smem, st);
}

template <class T>
void launch_backsub(Problem& P) {
  const Dims& d = P.d;
  BackArgs<T> a;
  a.fslot_off = P.fslot_off; a.slot_ent = P.slot_ent; a.slot_feat = P.slot_feat; a.feat_plane_slot = P.feat_plane_slot;
  a.slot_type = P.slot_type; a.V = P.featV; a.Vinv = P.featVinv; a.g = P.featg; a.x = P.x;
  a.W = (const T*)P.slotW; a.H = (const T*)P.slotH; a.G = (const T*)P.slotG; a.C = (const T*)P.slotC;
  a.sv = (T*)P.slotBS; a.df = P.dfeat; a.np = d.np; a.nf = d.nf; a.ne = d.ne; a.S = P.S; a.red = P.red;
  a.CK = (const T*)P.slotCK; a.cam_k = d.nk ? P.cam_k : nullptr; a.kbase = d.kbase(); a.CS = (const T*)P.slotCS;
  if (d.ne) { ++P.launches; k_backsub_slots<T><<<nblk(d.ne, 128), 128, 0, P.stream>>>(a); }
  ++P.launches;
  a.nfp = d.nfp;
  k_backsub<T><<<nblk(d.nfp > 0 ? d.nfp : 1, 128), 128, 0, P.stream>>>(a);
}

void launch_candidate(Problem& P) {
  const Dims& d = P.d;
  auto& c = P.ps[P.cur];
  auto& n = P.ps[1 - P.cur];
  CandArgs a;
  a.cam = c.cam; a.pts = c.pts; a.lin = c.lin; a.pln = c.pln; a.vps = c.vps; a.x = P.x; a.df = P.dfeat;
  a.fixed = P.cam_fixed; a.cam2 = n.cam; a.pts2 = n.pts; a.lin2 = n.lin; a.pln2 = n.pln; a.vps2 = n.vps;
  a.nc = d.nc; a.np = d.np; a.nl = d.nl; a.npl = d.npl; a.nv = d.nv;
  a.intr = c.intr; a.intr2 = n.intr; a.cam_k = P.cam_k; a.nk = d.nk; a.kbase = d.kbase();
  a.srf = c.srf; a.srf2 = n.srf; a.nsp = d.nsp; a.ncy = d.ncy; a.nco = d.nco; a.sbase = d.sbase();
  a.bx = c.bx; a.bx2 = n.bx; a.nel = d.nel; a.ncu = d.ncu; a.bbase = d.bbase();
  a.jq = d.njp ? P.jq : nullptr; a.jbase = d.jbase();
  int64_t tot = d.nc + d.npl + d.nv + d.np + d.nl + d.nk + d.ngs() + d.nbx();
  if (tot) { ++P.launches; k_candidate<<<nblk(tot, 128), 128, 0, P.stream>>>(a); }
}

void launch_cost(Problem& P, bool candidate) {
  const Dims& d = P.d;
  auto& s = P.ps[candidate ? 1 - P.cur : P.cur];
  CostArgs a;
  a.rkind = P.rkind; a.rcam = P.rcam; a.rfeat = P.rfeat; a.rgrp = P.rgrp; a.meas = P.meas64; a.order = P.cost_order;
  a.camD = s.camD; a.grpD = s.grpD; a.pts = s.pts; a.lin = s.lin; a.srf = s.srf; a.bx = s.bx;
  a.nr = d.nr_cost; a.np = d.np; a.npl = d.npl; a.nsp = d.nsp; a.ncy = d.ncy; a.nel = d.nel;
  a.partner = P.cost_partner;
  a.loss = make_loss(P.opt); a.S = P.S; a.red = P.red;
  a.candidate = candidate ? 1 : 0;
  ++P.launches;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, P.device) != cudaSuccess || sms <= 0) {
    cudaGetLastError();
    sms = 148;
  }
  const unsigned grid = (unsigned)std::min<int64_t>(nblk(d.nr > 0 ? d.nr : 1, 256), 2 * (int64_t)sms);
  if (d.ngs() || d.nbx() || d.njp) k_cost<true><<<grid, 256, 0, P.stream>>>(a);
  else k_cost<false><<<grid, 256, 0, P.stream>>>(a);
}

void launch_decide(Problem& P) {
  DecideArgs a{P.S, P.opt.min_gain, P.opt.lambda_min, P.opt.lambda_max};
  ++P.launches;
  k_decide<<<1, 1, 0, P.stream>>>(a);
}

// ============================================================================
// K10: many independent windows, one persistent launch
// ============================================================================
// Every window is a frozen problem of its own (structure, slots, S pattern, PCG chunking).  A CTA takes
// the next window from a queue (largest first) and runs all its LM iterations on the device: the same
// per-item bodies as the grid kernels above, strided over the CTA's threads, with CTA barriers between
// phases, a single-CTA PCG, and the accept / reject decision on thread 0.
template <class T>
struct WinDesc {
  int64_t nc, npl, nv, np, nl, nf, na, nr, nbu, nch;
  LinArgs<T> lin;
  InvArgs<T> inv;
  UnitArgs<T> units;
  BackArgs<T> back;
  CandArgs cand;
  CostArgs cost;
  DecideArgs dec;
  double *cam[2], *pts[2], *lin_[2], *pln[2], *vps[2], *camD[2], *grpD[2];
  T *camT, *grpT, *ptsT, *linT;
  const int32_t *row_ptr, *col, *row_chunk0, *chunk_beg;
  const T* Sval;
  T* Minv;
  const double* b;
  double *x, *r, *z, *p, *Ap;
  float2* phl;
  DevScalars* S;
  int* state;          // [0] current parameter set, [1] linearisation valid, [2] steps, [3] accepted, [4] converged
  double pcg_tol, rel_cost_tol;
  int pcg_max_iters;
};

// The CTAs that work on one window: a thread-block cluster of nct CTAs (nct = 1: a single CTA).  Every phase
// strides its items over the cluster's threads (or warps) and ends at a cluster barrier, which also orders the
// global-memory writes of one CTA before the reads of the others; the PCG's rows are split into nct contiguous
// ranges, one per CTA, so that a row's chunk sums stay in the shared memory of the CTA that formed them.
struct WinCtx {
  unsigned rank, nct;
  __device__ __forceinline__ int64_t t0() const { return (int64_t)rank * blockDim.x + threadIdx.x; }
  __device__ __forceinline__ int64_t ts() const { return (int64_t)nct * blockDim.x; }
  __device__ __forceinline__ int64_t w0() const { return (int64_t)rank * (blockDim.x >> 5) + (threadIdx.x >> 5); }
  __device__ __forceinline__ int64_t ws() const { return (int64_t)nct * (blockDim.x >> 5); }
  __device__ __forceinline__ void sync() const {
    if (nct == 1) __syncthreads();
    else cooperative_groups::this_cluster().sync();
  }
};

// cluster-wide sums of two values, the CTA sums added in rank order (identical in every CTA)
template <int NT>
__device__ __forceinline__ void win_sum2(const WinCtx& c, double v0, double v1, double* out2) {
  __shared__ double part[2];
  cta_sum2<NT>(v0, v1, part);
  if (c.nct == 1) {
    out2[0] = part[0];
    out2[1] = part[1];
    __syncthreads();
    return;
  }
  cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
  cl.sync();
  double a = 0, b = 0;
  for (unsigned r = 0; r < c.nct; ++r) {
    const double* q = cl.map_shared_rank(part, r);
    a += q[0];
    b += q[1];
  }
  cl.sync();   // every CTA has read the parts before any overwrites its own
  out2[0] = a;
  out2[1] = b;
  __syncthreads();
}

template <class T, int NT>
__device__ void window_pcg(const WinCtx& cx, const WinDesc<T>& W, double* chunk_mem, double* red2) {
  DotAcc<T>* chunk_y = reinterpret_cast<DotAcc<T>*>(chunk_mem);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = NT / 32;
  PcgArgs<T> a;
  a.p = W.p;
  a.phl = W.phl;
  const int64_t na = W.na;
  // this CTA's rows and their chunks
  const int64_t rb = na * cx.rank / cx.nct, re = na * (cx.rank + 1) / cx.nct;
  const int qb = W.row_chunk0[rb], qe = W.row_chunk0[re];
  double v0 = 0, v1 = 0;
  for (int64_t row = rb + threadIdx.x; row < re; row += NT) {
    double rv[6], zv[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) { rv[i] = W.b[6 * row + i]; W.x[6 * row + i] = 0; W.r[6 * row + i] = rv[i]; }
    apply_block(W.Minv + (size_t)row * BS2, rv, zv);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      W.z[6 * row + i] = zv[i];
      W.p[6 * row + i] = zv[i];
      if (W.phl) W.phl[6 * row + i] = split2(zv[i]);
      v0 += rv[i] * zv[i];
      v1 += rv[i] * rv[i];
    }
  }
  win_sum2<NT>(cx, v0, v1, red2);
  double rz = red2[0];
  const double bb = red2[1];
  const double tol2 = W.pcg_tol * W.pcg_tol * bb;
  double rr = bb;
  int it = 0;
  bool go = bb > 0;
  if (go) cx.sync();   // p of every row is written before any product reads it
  while (go) {
    for (int64_t q = qb + warp; q < qe; q += NW) {
      DotAcc<T> acc[6];
      const int blk = W.chunk_beg[q] + lane;
      T B[36];
      load_block36(W.Sval + s_idx(blk, 0), B);
      spmv_block(B, a, W.col[blk], acc);
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        const DotAcc<T> y = warp_sum_acc(acc[i]);
        if (lane == 0) chunk_y[6 * (q - qb) + i] = y;
      }
    }
    __syncthreads();
    double pap = 0;
    for (int64_t row = rb + threadIdx.x; row < re; row += NT) {
      DotAcc<T> y[6];
      for (int q = W.row_chunk0[row]; q < W.row_chunk0[row + 1]; ++q)
#pragma unroll
        for (int i = 0; i < 6; ++i) acc_add(y[i], chunk_y[6 * (q - qb) + i]);
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        const double yv = y[i].value();
        W.Ap[6 * row + i] = yv;
        pap += yv * W.p[6 * row + i];
      }
    }
    win_sum2<NT>(cx, pap, 0.0, red2);
    const double alpha = rz / red2[0];
    v0 = 0; v1 = 0;
    for (int64_t row = rb + threadIdx.x; row < re; row += NT) {
      double rv[6], zv[6];
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        W.x[6 * row + i] += alpha * W.p[6 * row + i];
        rv[i] = W.r[6 * row + i] - alpha * W.Ap[6 * row + i];
        W.r[6 * row + i] = rv[i];
      }
      apply_block(W.Minv + (size_t)row * BS2, rv, zv);
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        W.z[6 * row + i] = zv[i];
        v0 += rv[i] * rv[i];
        v1 += rv[i] * zv[i];
      }
    }
    win_sum2<NT>(cx, v0, v1, red2);
    rr = red2[0];
    const double rz_new = red2[1];
    ++it;
    if (rr <= tol2 || it >= W.pcg_max_iters || !(rr == rr)) break;
    const double beta = rz_new / rz;
    rz = rz_new;
    for (int64_t k = 6 * rb + threadIdx.x; k < 6 * re; k += NT) {
      const double pk = W.z[k] + beta * W.p[k];
      W.p[k] = pk;
      if (W.phl) W.phl[k] = split2(pk);
    }
    cx.sync();
  }
  if (cx.rank == 0 && threadIdx.x == 0) {
    W.S->iters = it;
    W.S->rr = rr;
    W.S->bnorm2 = bb;
  }
  cx.sync();
}

template <class T, int NT>
__device__ void window_step(const WinCtx& cx, const WinDesc<T>& W, double* chunk_y) {
  __shared__ double red2[2];
  __shared__ int s_cur, s_lin;
  if (threadIdx.x == 0) { s_cur = W.state[0]; s_lin = W.state[1]; }
  __syncthreads();
  const int cur = s_cur, nxt = 1 - s_cur;
  const bool flt = sizeof(T) == sizeof(float);
  const int64_t T0 = cx.t0(), TS = cx.ts();
  // ---- linearise at the current parameters (after an accepted step only)
  if (!s_lin) {
    for (int64_t i = T0; i < W.nc; i += TS) derive_cam<T>(W.cam[cur], W.camD[cur], flt ? W.camT : nullptr, i);
    for (int64_t i = T0; i < W.npl + W.nv; i += TS)
      derive_group<T>(W.npl, W.pln[cur], W.vps[cur], W.grpD[cur], flt ? W.grpT : nullptr, i);
    if (flt) {
      for (int64_t i = T0; i < 3 * W.np; i += TS) ((float*)W.ptsT)[i] = (float)W.pts[cur][i];
      for (int64_t i = T0; i < 6 * W.nl; i += TS) ((float*)W.linT)[i] = (float)W.lin_[cur][i];
    }
    cx.sync();
    LinArgs<T> la = W.lin;
    if (!flt) {
      la.cam = (const T*)W.camD[cur]; la.grp = (const T*)W.grpD[cur];
      la.pts = (const T*)W.pts[cur]; la.lin = (const T*)W.lin_[cur];
    }
    for (int64_t f = T0; f < W.np; f += TS) linearize_feature<T, 3>(la, f);
    for (int64_t f = W.np + T0; f < W.nf; f += TS) linearize_feature<T, 4>(la, f);
    cx.sync();
  }
  const double lam = W.S->lambda;
  // ---- damp + invert the landmark blocks, Schur complement, block-Jacobi
  {
    InvArgs<T> ia = W.inv;
    ia.lambda = lam;
    for (int64_t f = T0; f < W.nf; f += TS) {
      if (f < W.np) invert_feature<T, 3>(ia, f);
      else invert_feature<T, 4>(ia, f);
    }
  }
  cx.sync();
  {
    UnitArgs<T> ua = W.units;
    ua.fb.lambda = lam;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    char* mine = reinterpret_cast<char*>(chunk_y) + (size_t)warp * UnitSmem<T>::bytes;
    for (int64_t w = cx.w0(); w < ua.nun; w += cx.ws()) unit_warp<T>(ua, (int)w, mine, lane);
    cx.sync();
    for (int64_t k = T0; k < ua.nmulti; k += TS) unit_finish<T>(ua, ua.multi[k]);
  }
  cx.sync();
  for (int64_t r = T0; r < W.na; r += TS) precond_row<T, true>(W.row_ptr, W.col, W.Sval, W.Minv, W.S, r, SView());
  cx.sync();
  // ---- PCG, back-substitution and predicted decrease
  window_pcg<T, NT>(cx, W, chunk_y, red2);
  for (int64_t e = T0; e < W.back.ne; e += TS) backsub_slot<T>(W.back, e);
  cx.sync();
  double g = 0, h = 0;
  for (int64_t f = T0; f < W.nf; f += TS) {
    double gi = 0, hi = 0;
    if (f < W.np) backsub_feature<T, 3>(W.back, f, gi, hi);
    else backsub_feature<T, 4>(W.back, f, gi, hi);
    g += gi; h += hi;
  }
  win_sum2<NT>(cx, g, h, red2);
  if (cx.rank == 0 && threadIdx.x == 0) { W.S->gTd = red2[0]; W.S->dHd = red2[1]; W.S->pred = -red2[0] - 0.5 * red2[1]; }
  // ---- candidate, its FP64 cost, decision
  {
    CandArgs ca = W.cand;
    ca.cam = W.cam[cur]; ca.pts = W.pts[cur]; ca.lin = W.lin_[cur]; ca.pln = W.pln[cur]; ca.vps = W.vps[cur];
    ca.cam2 = W.cam[nxt]; ca.pts2 = W.pts[nxt]; ca.lin2 = W.lin_[nxt]; ca.pln2 = W.pln[nxt]; ca.vps2 = W.vps[nxt];
    const int64_t tot = W.nc + W.npl + W.nv + W.np + W.nl;
    for (int64_t i = T0; i < tot; i += TS) candidate_item(ca, i);
  }
  cx.sync();
  for (int64_t i = T0; i < W.nc; i += TS) derive_cam<T>(W.cam[nxt], W.camD[nxt], nullptr, i);
  for (int64_t i = T0; i < W.npl + W.nv; i += TS)
    derive_group<T>(W.npl, W.pln[nxt], W.vps[nxt], W.grpD[nxt], nullptr, i);
  cx.sync();
  {
    CostArgs co = W.cost;
    co.camD = W.camD[nxt]; co.grpD = W.grpD[nxt]; co.pts = W.pts[nxt]; co.lin = W.lin_[nxt];
    double e = 0, epx = 0;
    for (int64_t i = T0; i < W.nr; i += TS) {
      double v[2] = {0, 0};
      cost_residual(co, co.order[i], v);
      e += v[0]; epx += v[1];
    }
    win_sum2<NT>(cx, e, epx, red2);
  }
  if (cx.rank == 0 && threadIdx.x == 0) {
    DevScalars* S = W.S;
    S->Enew = red2[0];
    S->Epxnew = red2[1];
    const double lam_used = S->lambda;
    decide(W.dec);
    W.state[2] += 1;
    if (!S->accepted && lam_used >= W.dec.lmax && !W.state[4]) W.state[4] = W.state[2];   // no step helps any more
    if (S->accepted) {
      const double rel = fabs(S->Epx - S->Epxnew) / fmax(S->Epx, 1e-300);
      if (rel < W.rel_cost_tol && !W.state[4]) W.state[4] = W.state[2];
      S->E = S->Enew;
      S->Epx = S->Epxnew;
      W.state[0] = nxt;
      W.state[1] = 0;
      W.state[3] += 1;
    } else {
      W.state[1] = 1;
    }
  }
  cx.sync();
}

// The windows in `order` are sorted largest first.  Phase 1: a cluster of nct CTAs takes the next of the first
// nbig windows and runs its iterations together (rank 0 draws it from queue[0], the other CTAs read it from rank
// 0's shared memory).  Phase 2: once those are taken, every CTA on its own takes the next of the remaining
// windows from queue[1].  With nct = 1 (nbig = 0) every window runs on a single CTA.
template <class T, int NT>
__device__ __forceinline__ void run_window(const WinCtx& cx, const WinDesc<T>& W, int iters, double* chunk_y) {
  unsigned long long t0 = 0, t1 = 0;
  if (threadIdx.x == 0) asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (int it = 0; it < iters; ++it) window_step<T, NT>(cx, W, chunk_y);
  if (cx.rank == 0 && threadIdx.x == 0) {
    // the window's own device time on its CTAs (ns of the global timer), for the makespan report
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
    *reinterpret_cast<unsigned long long*>(W.state + 6) = t1 - t0;
  }
}

template <class T, int NT>
__global__ void __launch_bounds__(NT, 1) k_windows(const WinDesc<T>* __restrict__ descs, const int* __restrict__ order,
                                                   int nwin, int nbig, int iters, int* queue) {
  extern __shared__ __align__(16) double chunk_y[];
  __shared__ int s_w;
  const unsigned nct = cooperative_groups::this_cluster().num_blocks();
  if (nct > 1) {
    cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
    const WinCtx cx{cl.block_rank(), nct};
    for (;;) {
      if (cx.rank == 0 && threadIdx.x == 0) s_w = atomicAdd(&queue[0], 1);
      cl.sync();
      const int w = *cl.map_shared_rank(&s_w, 0);
      cl.sync();
      if (w >= nbig) break;
      run_window<T, NT>(cx, descs[order[w]], iters, chunk_y);
    }
  }
  const WinCtx solo{0u, 1u};
  for (;;) {
    if (threadIdx.x == 0) s_w = nbig + atomicAdd(&queue[1], 1);
    __syncthreads();
    const int w = s_w;
    __syncthreads();
    if (w >= nwin) break;
    run_window<T, NT>(solo, descs[order[w]], iters, chunk_y);
  }
}

template <class T>
void fill_window_desc(Problem& P, void* out) {
  WinDesc<T>& W = *(WinDesc<T>*)out;
  const Dims& d = P.d;
  W.nc = d.nc; W.npl = d.npl; W.nv = d.nv; W.np = d.np; W.nl = d.nl; W.nf = d.nf; W.na = d.na; W.nr = d.nr;
  W.nbu = d.nbu;
  std::vector<int32_t> rc(1);
  W.nch = 0;
  cudaMemcpy(&rc[0], P.row_chunk0 + d.na, sizeof(int32_t), cudaMemcpyDeviceToHost);
  W.nch = rc[0];
  const bool flt = sizeof(T) == sizeof(float);
  LinArgs<T>& a = W.lin;
  a.rkind = P.rkind; a.cam_mask = P.cam_fixed; a.rcam = P.rcam; a.rgrp = P.rgrp; a.rslot_c = P.rslot_c;
  a.rslot_g = P.rslot_g; a.fres_off = P.fres_off; a.feat_plane_slot = P.feat_plane_slot;
  a.meas = flt ? (const T*)P.measT : (const T*)P.meas64;
  a.cam = (const T*)P.camT; a.grp = (const T*)P.grpT; a.pts = (const T*)P.ptsT; a.lin = (const T*)P.linT;
  a.npl = d.npl; a.np = d.np;
  a.W = (T*)P.slotW; a.H = (T*)P.slotH; a.G = (T*)P.slotG; a.C = (T*)P.slotC; a.V = P.featV; a.g = P.featg;
  a.loss = make_loss(P.opt);
  a.rslot_k = nullptr; a.fslot_off = P.fslot_off; a.slot_type = P.slot_type; a.CK = nullptr;
  a.srf = nullptr; a.CS = nullptr; a.nsp = a.ncy = 0; a.bx = nullptr; a.nel = 0;
  a.jp_pt = nullptr; a.nf = d.nf;
  InvArgs<T>& ia = W.inv;
  ia.fslot_off = P.fslot_off; ia.V = P.featV; ia.g = P.featg; ia.W = (const T*)P.slotW; ia.G = (const T*)P.slotG;
  ia.slot_feat = P.slot_feat; ia.Vinv = P.featVinv; ia.u = P.featu; ia.L = P.featL; ia.Z = (T*)P.slotZ; ia.B = (T*)P.slotB;
  ia.np = d.np; ia.nf = d.nf; ia.ne = d.ne;
  ia.lambda = 0; ia.S = P.S;
  W.units = unit_args<T>(P, 0.0);
  BackArgs<T>& k = W.back;
  k.fslot_off = P.fslot_off; k.slot_ent = P.slot_ent; k.feat_plane_slot = P.feat_plane_slot; k.slot_type = P.slot_type;
  k.V = P.featV; k.Vinv = P.featVinv; k.g = P.featg; k.x = P.x; k.W = (const T*)P.slotW; k.H = (const T*)P.slotH;
  k.G = (const T*)P.slotG; k.C = (const T*)P.slotC; k.df = P.dfeat; k.np = d.np; k.nf = d.nf; k.S = P.S; k.red = P.red;
  k.slot_feat = P.slot_feat; k.sv = (T*)P.slotBS; k.ne = d.ne;
  k.CK = nullptr; k.cam_k = nullptr; k.kbase = 0; k.CS = nullptr; k.nfp = d.nf;
  CandArgs& c = W.cand;
  c.x = P.x; c.df = P.dfeat; c.fixed = P.cam_fixed; c.nc = d.nc; c.np = d.np; c.nl = d.nl; c.npl = d.npl; c.nv = d.nv;
  c.intr = nullptr; c.intr2 = nullptr; c.cam_k = nullptr; c.nk = 0; c.kbase = 0;   // windows: no refined intrinsics
  c.srf = nullptr; c.srf2 = nullptr; c.nsp = c.ncy = c.nco = 0; c.sbase = 0;        // nor surface groups
  c.bx = nullptr; c.bx2 = nullptr; c.nel = c.ncu = 0; c.bbase = 0;
  c.jq = nullptr; c.jbase = 0;                                                      // nor 3D wireframe distances
  CostArgs& co = W.cost;
  co.rkind = P.rkind; co.rcam = P.rcam; co.rfeat = P.rfeat; co.rgrp = P.rgrp; co.meas = P.meas64; co.order = P.cost_order;
  co.nr = d.nr; co.np = d.np; co.npl = d.npl; co.loss = make_loss(P.opt); co.S = P.S; co.red = P.red; co.candidate = 1;
  co.partner = nullptr;   // windows evaluate every record on its own
  co.srf = nullptr; co.nsp = co.ncy = 0; co.bx = nullptr; co.nel = 0;
  W.dec = DecideArgs{P.S, P.opt.min_gain, P.opt.lambda_min, P.opt.lambda_max};
  for (int s = 0; s < 2; ++s) {
    W.cam[s] = P.ps[s].cam; W.pts[s] = P.ps[s].pts; W.lin_[s] = P.ps[s].lin; W.pln[s] = P.ps[s].pln;
    W.vps[s] = P.ps[s].vps; W.camD[s] = P.ps[s].camD; W.grpD[s] = P.ps[s].grpD;
  }
  W.camT = (T*)P.camT; W.grpT = (T*)P.grpT; W.ptsT = (T*)P.ptsT; W.linT = (T*)P.linT;
  W.row_ptr = P.row_ptr; W.col = P.col; W.row_chunk0 = P.row_chunk0; W.chunk_beg = P.chunk_beg;
  W.Sval = (const T*)P.Sval; W.Minv = (T*)P.Minv; W.b = P.bvec; W.x = P.x; W.r = P.r; W.z = P.z; W.p = P.p;
  W.Ap = P.Ap; W.phl = flt ? P.phl : nullptr; W.S = P.S; W.state = P.win_state;
  W.pcg_tol = P.opt.pcg_rel_tol; W.rel_cost_tol = P.opt.rel_cost_tol; W.pcg_max_iters = P.opt.pcg_max_iters;
}

template <class T>
size_t window_desc_size() { return sizeof(WinDesc<T>); }

// dynamic shared memory of a window CTA: the PCG chunk sums (smem_pcg bytes, from the host) or the Schur
// stage areas of its warps, whichever is larger (the two phases never overlap)
template <class T, int NT>
size_t window_smem(size_t smem_pcg) {
  const size_t su = (size_t)(NT / 32) * UnitSmem<T>::bytes;
  return smem_pcg > su ? smem_pcg : su;
}

template <class T, int NT>
cudaError_t launch_windows_nt(cudaStream_t st, const void* descs, const int* order, int nwin, int nbig, int iters,
                              int* queue, int grid, size_t smem_pcg, int nct) {
  const size_t smem = window_smem<T, NT>(smem_pcg);
  cudaFuncSetAttribute(k_windows<T, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (nct > 1) cudaFuncSetAttribute(k_windows<T, NT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaError_t e = cudaMemsetAsync(queue, 0, 2 * sizeof(int), st);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)nct;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_windows<T, NT>, (const WinDesc<T>*)descs, order, nwin, nct > 1 ? nbig : 0, iters,
                            queue);
}

template <class T>
cudaError_t launch_windows(cudaStream_t st, const void* descs, const int* order, int nwin, int nbig, int iters,
                           int* queue, int threads, int grid, size_t smem, int nct) {
  if (threads == 128) return launch_windows_nt<T, 128>(st, descs, order, nwin, nbig, iters, queue, grid, smem, nct);
  return launch_windows_nt<T, 256>(st, descs, order, nwin, nbig, iters, queue, grid, smem, nct);
}

// clusters of nct window CTAs that can be resident at once (0 if the shape cannot launch)
template <class T, int NT>
int window_clusters_nt(size_t smem_pcg, int nct) {
  const size_t smem = window_smem<T, NT>(smem_pcg);
  cudaFuncSetAttribute(k_windows<T, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (nct > 1) cudaFuncSetAttribute(k_windows<T, NT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)nct);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)nct;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_windows<T, NT>, &cfg) != cudaSuccess) { cudaGetLastError(); return 0; }
  return n;
}

template <class T>
int window_clusters(int threads, size_t smem_pcg, int nct) {
  return threads == 128 ? window_clusters_nt<T, 128>(smem_pcg, nct) : window_clusters_nt<T, 256>(smem_pcg, nct);
}

template <class T, int NT>
int windows_per_sm_nt(size_t smem_pcg) {
  const size_t smem = window_smem<T, NT>(smem_pcg);
  cudaFuncSetAttribute(k_windows<T, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_windows<T, NT>, NT, smem);
  return nb;
}

template <class T>
int windows_per_sm(int threads, size_t smem_pcg) {
  return threads == 128 ? windows_per_sm_nt<T, 128>(smem_pcg) : windows_per_sm_nt<T, 256>(smem_pcg);
}

template void fill_window_desc<float>(Problem&, void*);
template void fill_window_desc<double>(Problem&, void*);
template size_t window_desc_size<float>();
template size_t window_desc_size<double>();
template cudaError_t launch_windows<float>(cudaStream_t, const void*, const int*, int, int, int, int*, int, int, size_t, int);
template cudaError_t launch_windows<double>(cudaStream_t, const void*, const int*, int, int, int, int*, int, int, size_t, int);
template int window_clusters<float>(int, size_t, int);
template int window_clusters<double>(int, size_t, int);
template int windows_per_sm<float>(int, size_t);
template int windows_per_sm<double>(int, size_t);

#define INST(T)                                         \
  template void launch_prepare<T>(Problem&, bool, bool); \
  template void launch_linearize<T>(Problem&);          \
  template void launch_invert<T>(Problem&, double);     \
  template void launch_schur<T>(Problem&, double);      \
  template void launch_precond<T>(Problem&);            \
  template void launch_pcg<T>(Problem&);                \
  template int pcg_blocks_per_sm<T>(size_t);            \
  template void pcg_allow_smem<T>(size_t);              \
  template size_t pcg_typed_fixed_smem<T>(int);         \
  template size_t pcg_typed_gacc_bytes<T>(int);         \
  template int pcg_typed_blocks_per_sm<T>(size_t);      \
  template void launch_backsub<T>(Problem&);
INST(double)
INST(float)

}  // namespace ba
