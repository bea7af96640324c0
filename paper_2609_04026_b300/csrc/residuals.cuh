// Residuals and analytic Jacobians of the seven residual kinds of holistic BA.
//
// Every function is templated on the arithmetic type T (double for the FP64
// path, float for the mixed path) and on JAC (false: value only, used by the
// FP64 cost pass).  Jacobians are taken with respect to the minimal local
// increments of each parameter block:
//   camera pose  R <- Exp(dw) R, t <- t + dt                       (6)
//   point        X <- X + dX                                        (3)
//   line         orthonormal (Bartoli-Sturm) update of Pluecker (d, m), |d| = 1:
//                U = [m/|m|, d, u1 x d] <- U Exp(dl0..2), phi <- phi + dl3,
//                d = u2, m = cot(phi) u1                            (4)
//   plane (n,w)  n <- Exp_n(b1 dg0 + b2 dg1) on S^2, w <- w + dg2    (3)
//   VP v         v <- Exp_v(b1 dg0 + b2 dg1)                        (2)
// with (b1, b2) the tangent basis: a = e_x unless |n_x| >= 0.9 (then e_y),
// b1 = unit(a - (a.n) n), b2 = n x b1.
//
// Residuals (Section 3 of the paper):
//   R1 point reprojection       Eq. 1 / Eq. 4, radial distortion (f, k1, k2)
//   R2 line reprojection        Eq. 4, rho = perpendicular displacement vectors
//   R3 plane-induced point      Eq. 7, plane projection of Appendix B
//   R4 plane-induced line       Eq. 8, Pluecker plane projection of Appendix B
//   R5 VP angular               Eq. 6 written as the 3-vector d x v
//   R6 wireframe point->line    Eq. 11 (pinhole pixels)
//   R7 wireframe line->point    Eq. 12 (pinhole pixels)
//   sphere / cylinder / cone point residuals: Eq. 7 with the projections of Appendix B (radial onto a sphere;
//   radial about a cylinder's axis; onto a cone along the normal of its generatrix)
//   3D point-to-plane and line-to-plane distances: the direct 3D form of the plane constraint that Section 3.2
//   sets against the group-induced residuals (Table 5 weighs it); no camera, not in the pixel cost
// Lines and the wireframe terms live in undistorted pixel coordinates; only R1
// and R3 use k1, k2.
// With INTR (refined intrinsics, Section 3.1) a residual also gives its rows of the
// Jacobian with respect to the additive increments of the camera's (f, k1, k2).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ba {

enum ResKind : int {
  R_POINT = 0, R_LINE = 1, R_PLANE_POINT = 2, R_PLANE_LINE = 3, R_VP = 4, R_P2L = 5, R_L2P = 6,
  R_PLANE_POINT3 = 7, R_PLANE_LINE3 = 8,   // the direct 3D plane distances (no camera)
  R_SPHERE_POINT = 9, R_CYL_POINT = 10, R_CONE_POINT = 11,  // group-induced point residuals of other group types
  R_ELL_POINT = 12, R_CUB_POINT = 13,                        // ... of the 9-parameter ellipsoid and cuboid
  R_WF3D = 14,                                               // 3D wireframe endpoint distance (line, point)
  R_CUB_LINE = 15                                            // Eq. 8 onto a cuboid's face (Appendix B)
};
constexpr int N_KINDS = 16;

__host__ __device__ constexpr int res_dim(int k) {
  return k == R_POINT ? 2 : k == R_LINE ? 4 : k == R_PLANE_POINT ? 2 : k == R_PLANE_LINE ? 4 : k == R_VP ? 3
       : k == R_PLANE_LINE3 ? 2 : k == R_WF3D ? 3 : k == R_CUB_LINE ? 4 : k >= R_SPHERE_POINT ? 2 : 1;
}
// surface group types (sphere, cylinder, cone): 8 raw values per group, increments of 4, 5 and 6
constexpr int SRF_STRIDE = 8;
// 9-parameter groups (ellipsoid, cuboid): R row-major (9) then (c, s) or the six face offsets; two entities each
// (rotation and c or d_0..2; then log s or d_3..5)
constexpr int BOX_STRIDE = 16;
__host__ __device__ constexpr int srf_dims(int ty) { return ty == 0 ? 4 : (ty == 1 ? 5 : 6); }
// kinds with a camera (the others: the VP term and the direct 3D plane distances)
__host__ __device__ constexpr bool res_has_cam(int k) {
  return k != R_VP && k != R_PLANE_POINT3 && k != R_PLANE_LINE3 && k != R_WF3D;
}
// kinds in the pixel cost E_px
__host__ __device__ constexpr bool res_pixel(int k) { return res_has_cam(k); }

// per-camera data precomputed from the FP64 master parameters each time they change
// layout (stride CAM_STRIDE): R row-major (9), t (3), f, k1, k2, ppx, ppy
constexpr int CAM_STRIDE = 20;
// per-plane data: n (3), w, b1 (3), b2 (3) ; per-VP data: v (3), 0, b1 (3), b2 (3)
constexpr int GRP_STRIDE = 12;

template <class T>
struct Cam {
  T R[9], t[3], f, k1, k2, px, py;
};

// a camera record (CAM_STRIDE elements, 16-byte aligned); the float records of the linearisation are read
// with 16-byte loads, the FP64 ones element by element (the FP64 cost pass runs faster with fewer values live)
template <class T>
__device__ __forceinline__ void load_cam(const T* __restrict__ c, Cam<T>& o) {
  if constexpr (sizeof(T) == 4) {
    T v[20];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const float4 q = reinterpret_cast<const float4*>(c)[k];
      v[4 * k] = q.x; v[4 * k + 1] = q.y; v[4 * k + 2] = q.z; v[4 * k + 3] = q.w;
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) o.R[i] = v[i];
    o.t[0] = v[9]; o.t[1] = v[10]; o.t[2] = v[11];
    o.f = v[12]; o.k1 = v[13]; o.k2 = v[14]; o.px = v[15]; o.py = v[16];
  } else {
#pragma unroll
    for (int i = 0; i < 9; ++i) o.R[i] = c[i];
    o.t[0] = c[9]; o.t[1] = c[10]; o.t[2] = c[11];
    o.f = c[12]; o.k1 = c[13]; o.k2 = c[14]; o.px = c[15]; o.py = c[16];
  }
}

template <class T> __device__ __forceinline__ T dot3(const T* a, const T* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
template <class T> __device__ __forceinline__ void cross3(const T* a, const T* b, T* o) {
  T x = a[1] * b[2] - a[2] * b[1], y = a[2] * b[0] - a[0] * b[2], z = a[0] * b[1] - a[1] * b[0];
  o[0] = x; o[1] = y; o[2] = z;
}
template <class T> __device__ __forceinline__ void matvec3(const T* R, const T* v, T* o) {
  T x = R[0] * v[0] + R[1] * v[1] + R[2] * v[2];
  T y = R[3] * v[0] + R[4] * v[1] + R[5] * v[2];
  T z = R[6] * v[0] + R[7] * v[1] + R[8] * v[2];
  o[0] = x; o[1] = y; o[2] = z;
}
template <class T> __device__ __forceinline__ T rsqrt_t(T x);
template <> __device__ __forceinline__ double rsqrt_t<double>(double x) { return 1.0 / sqrt(x); }
template <> __device__ __forceinline__ float rsqrt_t<float>(float x) { return 1.0f / sqrtf(x); }
template <class T> __device__ __forceinline__ T sqrt_t(T x);
template <> __device__ __forceinline__ double sqrt_t<double>(double x) { return sqrt(x); }
template <> __device__ __forceinline__ float sqrt_t<float>(float x) { return sqrtf(x); }

// Output of one residual: r (rd values) and Jacobian rows w.r.t. camera (6),
// feature (3 or 4) and group (3; VP uses the first 2).
template <class T>
struct ResJ {
  T r[4];
  T Jc[4][6];
  T Jf[4][4];
  T Jg[4][6];   // w.r.t. the group's increments (plane 3, VP 2, sphere 4, cylinder 5, cone 6; a 9-parameter
                // group's first entity 6)
  T Jg2[4][3];  // w.r.t. a 9-parameter group's second entity (ellipsoid log semi-axes, cuboid d_3..5)
  T Jk[4][3];   // w.r.t. the camera's (f, k1, k2), filled only when asked for (INTR)
  bool valid;
};

// d pi / d (f, k1, k2) of the distorted projection of x_cam: (s u, f r^2 u, f r^4 u), the same with v
template <class T>
__device__ __forceinline__ void project_dist_k(const Cam<T>& c, const T* xc, T Jk[2][3]) {
  T iz = T(1) / xc[2];
  T u = xc[0] * iz, v = xc[1] * iz;
  T r2 = u * u + v * v;
  T s = T(1) + c.k1 * r2 + c.k2 * r2 * r2;
  T fr2 = c.f * r2, fr4 = c.f * r2 * r2;
  Jk[0][0] = s * u; Jk[0][1] = fr2 * u; Jk[0][2] = fr4 * u;
  Jk[1][0] = s * v; Jk[1][1] = fr2 * v; Jk[1][2] = fr4 * v;
}

// ---------------------------------------------------------------- camera / point pieces
// rotation columns of the pose Jacobian for one row g of d(res)/d(x_cam):
//   d x_cam / d dw = -[R X]x  =>  row contribution  (R X) x g ; translation part = g
template <class T>
__device__ __forceinline__ void pose_row_point(const T* p, const T* g, T* out6) {
  T c[3];
  cross3(p, g, c);
  out6[0] = c[0]; out6[1] = c[1]; out6[2] = c[2];
  out6[3] = g[0]; out6[4] = g[1]; out6[5] = g[2];
}

// distorted projection of x_cam: pi = pp + f s (u, v); Jxc = d pi / d x_cam (2x3)
template <class T, bool JAC>
__device__ __forceinline__ void project_dist(const Cam<T>& c, const T* xc, T* pi, T Jxc[2][3]) {
  T iz = T(1) / xc[2];
  T u = xc[0] * iz, v = xc[1] * iz;
  T r2 = u * u + v * v;
  T s = T(1) + c.k1 * r2 + c.k2 * r2 * r2;
  pi[0] = c.px + c.f * s * u;
  pi[1] = c.py + c.f * s * v;
  if (JAC) {
    T ds = T(2) * (c.k1 + T(2) * c.k2 * r2);
    T a00 = c.f * (s + ds * u * u), a01 = c.f * ds * u * v, a11 = c.f * (s + ds * v * v);
    // d(u,v)/d x_cam = iz [[1,0,-u],[0,1,-v]]
    Jxc[0][0] = a00 * iz; Jxc[0][1] = a01 * iz; Jxc[0][2] = -(a00 * u + a01 * v) * iz;
    Jxc[1][0] = a01 * iz; Jxc[1][1] = a11 * iz; Jxc[1][2] = -(a01 * u + a11 * v) * iz;
  }
}

template <class T, bool JAC>
__device__ __forceinline__ void project_pin(const Cam<T>& c, const T* xc, T* pi, T Jxc[2][3]) {
  T iz = T(1) / xc[2];
  T u = xc[0] * iz, v = xc[1] * iz;
  pi[0] = c.px + c.f * u;
  pi[1] = c.py + c.f * v;
  if (JAC) {
    T fz = c.f * iz;
    Jxc[0][0] = fz; Jxc[0][1] = 0; Jxc[0][2] = -fz * u;
    Jxc[1][0] = 0; Jxc[1][1] = fz; Jxc[1][2] = -fz * v;
  }
}

// ---------------------------------------------------------------- line pieces
// orthonormal frame of a Pluecker line with |d| = 1: u1 = m/|m| (or the tangent
// basis vector b1(d) when |m| ~ 0), u3 = u1 x d, r = |m|
template <class T>
__device__ __forceinline__ void tangent_b1(const T* n, T* b1) {
  T a[3] = {T(0), T(0), T(0)};
  if (fabs(n[0]) < T(0.9)) a[0] = T(1); else a[1] = T(1);
  T an = dot3(a, n);
  b1[0] = a[0] - an * n[0]; b1[1] = a[1] - an * n[1]; b1[2] = a[2] - an * n[2];
  T s = rsqrt_t(dot3(b1, b1));
  b1[0] *= s; b1[1] *= s; b1[2] *= s;
}

template <class T>
__device__ __forceinline__ void line_frame(const T* d, const T* m, T* u1, T* u3, T& r) {
  r = sqrt_t(dot3(m, m));
  if (r < T(1e-12)) {
    tangent_b1(d, u1);
  } else {
    T ir = T(1) / r;
    u1[0] = m[0] * ir; u1[1] = m[1] * ir; u1[2] = m[2] * ir;
  }
  cross3(u1, d, u3);
}

// partial derivatives of (d, m) w.r.t. the 4 line increments, as directions:
//   dd/dl = [u3, 0, -u1, 0],  dm/dl = [0, -r u3, r u2, -(1 + r^2) u1]   (u2 = d)
template <class T>
__device__ __forceinline__ void line_dirs(const T* d, const T* u1, const T* u3, T r, T dd[4][3], T dm[4][3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    dd[0][i] = u3[i]; dd[1][i] = 0; dd[2][i] = -u1[i]; dd[3][i] = 0;
    dm[0][i] = 0; dm[1][i] = -r * u3[i]; dm[2][i] = r * d[i]; dm[3][i] = -(T(1) + r * r) * u1[i];
  }
}

// camera-frame moment m_c = R m + t x (R d), d_c = R d; image line l = K_l m_c
template <class T>
__device__ __forceinline__ void line_to_cam(const Cam<T>& c, const T* d, const T* m, T* dc, T* Rm, T* mc) {
  matvec3(c.R, d, dc);
  matvec3(c.R, m, Rm);
  T tx[3];
  cross3(c.t, dc, tx);
  mc[0] = Rm[0] + tx[0]; mc[1] = Rm[1] + tx[1]; mc[2] = Rm[2] + tx[2];
}

template <class T>
__device__ __forceinline__ void image_line(const Cam<T>& c, const T* mc, T* l) {
  l[0] = mc[0]; l[1] = mc[1]; l[2] = c.f * mc[2] - c.px * mc[0] - c.py * mc[1];
}

// rho(l, seg) (Eq. 4): per endpoint e, v_e = (l . [e;1]) (l0,l1) / |(l0,l1)|^2.
// J (4x3) = d rho / d l, then G = J K_l (chain to m_c).  Returns |(l0,l1)|^2.
template <class T, bool JAC>
__device__ __forceinline__ T rho_line(const Cam<T>& c, const T* l, const T* seg, T* r4, T G[4][3]) {
  T A2 = l[0] * l[0] + l[1] * l[1];
  T iA = T(1) / A2;
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    T ex = seg[2 * e], ey = seg[2 * e + 1];
    T q = l[0] * ex + l[1] * ey + l[2];
    T s = q * iA;
    r4[2 * e] = s * l[0];
    r4[2 * e + 1] = s * l[1];
    if (JAC) {
      T k = T(2) * q * iA * iA;
      T J[2][3];
      // d v / d l0 = (ex a + q e0)/A2 - 2 q l0 a / A2^2, similarly l1; d v / d l2 = a / A2
      J[0][0] = (ex * l[0] + q) * iA - k * l[0] * l[0];
      J[1][0] = (ex * l[1]) * iA - k * l[0] * l[1];
      J[0][1] = (ey * l[0]) * iA - k * l[1] * l[0];
      J[1][1] = (ey * l[1] + q) * iA - k * l[1] * l[1];
      J[0][2] = l[0] * iA;
      J[1][2] = l[1] * iA;
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        G[2 * e + i][0] = J[i][0] - c.px * J[i][2];
        G[2 * e + i][1] = J[i][1] - c.py * J[i][2];
        G[2 * e + i][2] = c.f * J[i][2];
      }
    }
  }
  return A2;
}

// for one row g (3) of d(res)/d(m_c): pose columns of a line with camera-frame
// direction dc and rotated moment Rm:  rot = Rm x g + dc x (g x t),  trans = dc x g
template <class T>
__device__ __forceinline__ void pose_row_line(const Cam<T>& c, const T* dc, const T* Rm, const T* g, T* out6) {
  T a[3], gt[3], b[3], tr[3];
  cross3(Rm, g, a);
  cross3(g, c.t, gt);
  cross3(dc, gt, b);
  cross3(dc, g, tr);
  out6[0] = a[0] + b[0]; out6[1] = a[1] + b[1]; out6[2] = a[2] + b[2];
  out6[3] = tr[0]; out6[4] = tr[1]; out6[5] = tr[2];
}

// d m_c along a perturbation (zeta of d, mu of m):  t x (R zeta) + R mu
template <class T>
__device__ __forceinline__ void dmc_dir(const Cam<T>& c, const T* zeta, const T* mu, T* o) {
  T Rz[3], Rmu[3], tx[3];
  matvec3(c.R, zeta, Rz);
  matvec3(c.R, mu, Rmu);
  cross3(c.t, Rz, tx);
  o[0] = tx[0] + Rmu[0]; o[1] = tx[1] + Rmu[1]; o[2] = tx[2] + Rmu[2];
}

// ---------------------------------------------------------------- plane projections (Appendix B)
template <class T>
__device__ __forceinline__ void plane_proj_point(const T* n, T w, const T* X, T* Xp, T& cdist) {
  cdist = dot3(n, X) + w;
  Xp[0] = X[0] - cdist * n[0]; Xp[1] = X[1] - cdist * n[1]; Xp[2] = X[2] - cdist * n[2];
}

// d' = d - (d.n) n ; m' = (1 - a^2/|d|^2) m + (a g/|d|^2) d + (w - dl/|d|^2)(d x n)
template <class T>
__device__ __forceinline__ void plane_proj_line(const T* n, T w, const T* d, const T* m, T* dp, T* mp) {
  T a = dot3(d, n), g = dot3(m, n), dd = dot3(d, d);
  T dxn[3];
  cross3(d, n, dxn);
  T dl = dot3(dxn, m);
  T idd = T(1) / dd;
  T A = T(1) - a * a * idd, B = a * g * idd, C = w - dl * idd;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    dp[i] = d[i] - a * n[i];
    mp[i] = A * m[i] + B * d[i] + C * dxn[i];
  }
}

// directional derivative of (d', m') for perturbations zeta (of d), mu (of m),
// eta (of n) and dw (of w)
template <class T>
__device__ __forceinline__ void plane_proj_line_dir(const T* n, T w, const T* d, const T* m, const T* zeta,
                                                    const T* mu, const T* eta, T dw, T* ddp, T* dmp) {
  T a = dot3(d, n), g = dot3(m, n), dd = dot3(d, d);
  T dxn[3];
  cross3(d, n, dxn);
  T dl = dot3(dxn, m);
  T idd = T(1) / dd;
  T A = T(1) - a * a * idd, B = a * g * idd, C = w - dl * idd;
  // first-order changes of the scalars
  T da = dot3(zeta, n) + dot3(d, eta);
  T dg = dot3(mu, n) + dot3(m, eta);
  T zxn[3], dxe[3];
  cross3(zeta, n, zxn);
  cross3(d, eta, dxe);
  T ddxn[3] = {zxn[0] + dxe[0], zxn[1] + dxe[1], zxn[2] + dxe[2]};
  T ddl = dot3(ddxn, m) + dot3(dxn, mu);
  T ddd = T(2) * dot3(d, zeta);
  T dA = -(T(2) * a * da) * idd + a * a * ddd * idd * idd;
  T dB = (da * g + a * dg) * idd - a * g * ddd * idd * idd;
  T dC = dw - ddl * idd + dl * ddd * idd * idd;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    ddp[i] = zeta[i] - da * n[i] - a * eta[i];
    dmp[i] = dA * m[i] + A * mu[i] + dB * d[i] + B * zeta[i] + dC * dxn[i] + C * ddxn[i];
  }
}

// ---------------------------------------------------------------- the seven residuals
// R1: pi(C, X) - x_ij
template <class T, bool JAC, bool INTR = false>
__device__ void res_point(const Cam<T>& c, const T* X, const T* meas, ResJ<T>& o) {
  T p[3], xc[3], pi[2], J[2][3];
  matvec3(c.R, X, p);
  xc[0] = p[0] + c.t[0]; xc[1] = p[1] + c.t[1]; xc[2] = p[2] + c.t[2];
  o.valid = xc[2] > T(1e-6);
  if (!o.valid) return;
  project_dist<T, JAC>(c, xc, pi, J);
  o.r[0] = pi[0] - meas[0];
  o.r[1] = pi[1] - meas[1];
  if (JAC) {
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      pose_row_point(p, J[i], o.Jc[i]);
      // d/dX = J R
#pragma unroll
      for (int k = 0; k < 3; ++k) o.Jf[i][k] = J[i][0] * c.R[k] + J[i][1] * c.R[3 + k] + J[i][2] * c.R[6 + k];
    }
    if (INTR) project_dist_k(c, xc, o.Jk);
  }
}

// R2: rho(pi_l(C, L), segment)
template <class T, bool JAC, bool INTR = false>
__device__ void res_line(const Cam<T>& c, const T* L, const T* seg, ResJ<T>& o) {
  T dc[3], Rm[3], mc[3], l[3], G[4][3];
  line_to_cam(c, L, L + 3, dc, Rm, mc);
  image_line(c, mc, l);
  T A2 = rho_line<T, JAC>(c, l, seg, o.r, G);
  o.valid = A2 > T(1e-24);
  if (!JAC || !o.valid) return;
  T u1[3], u3[3], r;
  line_frame(L, L + 3, u1, u3, r);
  T ddir[4][3], mdir[4][3], dmc[4][3];
  line_dirs(L, u1, u3, r, ddir, mdir);
#pragma unroll
  for (int k = 0; k < 4; ++k) dmc_dir(c, ddir[k], mdir[k], dmc[k]);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    pose_row_line(c, dc, Rm, G[i], o.Jc[i]);
#pragma unroll
    for (int k = 0; k < 4; ++k) o.Jf[i][k] = dot3(G[i], dmc[k]);
  }
  if (INTR) {
    // only l_2 = f m_c2 - ... depends on f (d l_2 / d f = m_c2), and d rho / d l_2 = (l0, l1) / |l_12|^2 at
    // both endpoints; the line terms are undistorted
    const T a = mc[2] / A2;
#pragma unroll
    for (int i = 0; i < 4; ++i) { o.Jk[i][0] = l[i & 1] * a; o.Jk[i][1] = 0; o.Jk[i][2] = 0; }
  }
}

// R3: pi(C, X) - pi(C, Proj_plane(X))  (Eq. 7)
template <class T, bool JAC, bool INTR = false>
__device__ void res_plane_point(const Cam<T>& c, const T* X, const T* P, ResJ<T>& o) {
  const T* n = P;
  T w = P[3];
  T Xp[3], cd;
  plane_proj_point(n, w, X, Xp, cd);
  T p1[3], p2[3], x1[3], x2[3], pi1[2], pi2[2], J1[2][3], J2[2][3];
  matvec3(c.R, X, p1);
  matvec3(c.R, Xp, p2);
#pragma unroll
  for (int i = 0; i < 3; ++i) { x1[i] = p1[i] + c.t[i]; x2[i] = p2[i] + c.t[i]; }
  o.valid = x1[2] > T(1e-6) && x2[2] > T(1e-6);
  if (!o.valid) return;
  project_dist<T, JAC>(c, x1, pi1, J1);
  project_dist<T, JAC>(c, x2, pi2, J2);
  o.r[0] = pi1[0] - pi2[0];
  o.r[1] = pi1[1] - pi2[1];
  if (JAC) {
    const T* b1 = P + 4;
    const T* b2 = P + 7;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      T a6[6], b6[6];
      pose_row_point(p1, J1[i], a6);
      pose_row_point(p2, J2[i], b6);
#pragma unroll
      for (int k = 0; k < 6; ++k) o.Jc[i][k] = a6[k] - b6[k];
      // g1 = J1 R, g2 = J2 R  (rows as 3-vectors in world frame)
      T g1[3], g2[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        g1[k] = J1[i][0] * c.R[k] + J1[i][1] * c.R[3 + k] + J1[i][2] * c.R[6 + k];
        g2[k] = J2[i][0] * c.R[k] + J2[i][1] * c.R[3 + k] + J2[i][2] * c.R[6 + k];
      }
      // d Xp / d X = I - n n^T
      T g2n = dot3(g2, n);
#pragma unroll
      for (int k = 0; k < 3; ++k) o.Jf[i][k] = g1[k] - (g2[k] - g2n * n[k]);
      // d Xp along eta (of n) = -((X.eta) n + cd eta);  along w: -n
      T gX = dot3(g2, X);
      (void)gX;
      T e1 = dot3(X, b1), e2 = dot3(X, b2);
      o.Jg[i][0] = (e1 * g2n + cd * dot3(g2, b1));
      o.Jg[i][1] = (e2 * g2n + cd * dot3(g2, b2));
      o.Jg[i][2] = g2n;
    }
    if (INTR) {
      T K1[2][3], K2[2][3];
      project_dist_k(c, x1, K1);
      project_dist_k(c, x2, K2);
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) o.Jk[i][k] = K1[i][k] - K2[i][k];
    }
  }
}

// R4: rho(pi_l(C, L)) - rho(pi_l(C, Proj_plane(L)))  (Eq. 8)
// Eq. 8 for the plane (n, w): r, Jc, Jf (and Jk); the group columns through gdir(k, dn, dw), the plane change of
// column k (normal change dn, offset change dw), stored by gput(i, k, value), for NG columns
template <class T, bool JAC, bool INTR, int NG, class GDir, class GPut>
__device__ __forceinline__ void plane_line_core(const Cam<T>& c, const T* L, const T* n, T w, const T* seg, ResJ<T>& o,
                                                GDir gdir, GPut gput) {
  const T* d = L;
  const T* m = L + 3;
  T dp[3], mp[3];
  plane_proj_line(n, w, d, m, dp, mp);
  T dc1[3], Rm1[3], mc1[3], l1[3], G1[4][3], r1[4];
  T dc2[3], Rm2[3], mc2[3], l2[3], G2[4][3], r2[4];
  line_to_cam(c, d, m, dc1, Rm1, mc1);
  line_to_cam(c, dp, mp, dc2, Rm2, mc2);
  image_line(c, mc1, l1);
  image_line(c, mc2, l2);
  T A1 = rho_line<T, JAC>(c, l1, seg, r1, G1);
  T A2 = rho_line<T, JAC>(c, l2, seg, r2, G2);
  o.valid = A1 > T(1e-24) && A2 > T(1e-24);
  if (!o.valid) return;
#pragma unroll
  for (int i = 0; i < 4; ++i) o.r[i] = r1[i] - r2[i];
  if (!JAC) return;
  T u1[3], u3[3], r;
  line_frame(d, m, u1, u3, r);
  T ddir[4][3], mdir[4][3], dmc1[4][3], dmc2[4][3];
  line_dirs(d, u1, u3, r, ddir, mdir);
  const T zero3[3] = {T(0), T(0), T(0)};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    dmc_dir(c, ddir[k], mdir[k], dmc1[k]);
    T ddp[3], dmp[3];
    plane_proj_line_dir(n, w, d, m, ddir[k], mdir[k], zero3, T(0), ddp, dmp);
    dmc_dir(c, ddp, dmp, dmc2[k]);
  }
  T dmcg[NG][3];
#pragma unroll
  for (int k = 0; k < NG; ++k) {
    T dn[3], dw, ddp[3], dmp[3];
    gdir(k, dn, dw);
    plane_proj_line_dir(n, w, d, m, zero3, zero3, dn, dw, ddp, dmp);
    dmc_dir(c, ddp, dmp, dmcg[k]);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    T a6[6], b6[6];
    pose_row_line(c, dc1, Rm1, G1[i], a6);
    pose_row_line(c, dc2, Rm2, G2[i], b6);
#pragma unroll
    for (int k = 0; k < 6; ++k) o.Jc[i][k] = a6[k] - b6[k];
#pragma unroll
    for (int k = 0; k < 4; ++k) o.Jf[i][k] = dot3(G1[i], dmc1[k]) - dot3(G2[i], dmc2[k]);
#pragma unroll
    for (int k = 0; k < NG; ++k) gput(i, k, -dot3(G2[i], dmcg[k]));
  }
  if (INTR) {
    const T a1 = mc1[2] / A1, a2 = mc2[2] / A2;
#pragma unroll
    for (int i = 0; i < 4; ++i) { o.Jk[i][0] = l1[i & 1] * a1 - l2[i & 1] * a2; o.Jk[i][1] = 0; o.Jk[i][2] = 0; }
  }
}

// R4: Eq. 8 with the plane (n, w) and its tangent basis b1, b2 (P + 4, P + 7): group columns b1, b2 (normal), w
template <class T, bool JAC, bool INTR = false>
__device__ void res_plane_line(const Cam<T>& c, const T* L, const T* P, const T* seg, ResJ<T>& o) {
  plane_line_core<T, JAC, INTR, 3>(
      c, L, P, P[3], seg, o,
      [&](int k, T* dn, T& dw) {
        const T* b = k == 0 ? P + 4 : P + 7;
#pragma unroll
        for (int i = 0; i < 3; ++i) dn[i] = k < 2 ? b[i] : T(0);
        dw = k == 2 ? T(1) : T(0);
      },
      [&](int i, int k, T v) { o.Jg[i][k] = v; });
}

// R5: d x v (Eq. 6 as a 3-vector; |d| = 1)
template <class T, bool JAC, bool INTR = false>
__device__ void res_vp(const T* L, const T* V, ResJ<T>& o) {
  const T* d = L;
  T dn = rsqrt_t(dot3(d, d));
  T dh[3] = {d[0] * dn, d[1] * dn, d[2] * dn};
  const T* v = V;
  cross3(dh, v, o.r);
  o.valid = true;
  if (!JAC) return;
  T u1[3], u3[3], r;
  line_frame(L, L + 3, u1, u3, r);
  // d(d x v)/d d = -[v]x ; increments of d: [u3, 0, -u1, 0] (all orthogonal to d)
  T c0[3], c2[3];
  cross3(u3, v, c0);
  cross3(u1, v, c2);
  const T* b1 = V + 4;
  const T* b2 = V + 7;
  T g0[3], g1[3];
  cross3(dh, b1, g0);
  cross3(dh, b2, g1);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    o.Jf[i][0] = c0[i] * dn; o.Jf[i][1] = 0; o.Jf[i][2] = -c2[i] * dn; o.Jf[i][3] = 0;
    o.Jg[i][0] = g0[i]; o.Jg[i][1] = g1[i]; o.Jg[i][2] = 0;
#pragma unroll
    for (int k = 0; k < 6; ++k) o.Jc[i][k] = 0;
    if (INTR) { o.Jk[i][0] = 0; o.Jk[i][1] = 0; o.Jk[i][2] = 0; }
  }
}

// ---------------------------------------------------------------- sphere, cylinder, cone (Appendix B)
// Projection Xp of X onto the surface and its directional derivative dXp for a change dX of X and a change of
// the group along increment k (k < 0: none).  Sphere (c, r): Xp = c + r u/|u|, u = X - c; increments dc (3),
// d log r.  Cylinder (axis d, m with |d| = 1, radius r): foot p0 = d x m, v = X - p0, Xp = p0 + (v.d) d + r w/|w|
// with w the radial part of v; increments: the line update of the axis (4), d log r.  Cone (apex a, unit axis
// d, half-angle al): v = X - a, e the radial unit of v, generatrix g = cos(al) d + sin(al) e, Xp = a + (v.g) g;
// increments da (3), the axis along the tangent basis (2), d al.
template <class T>
struct SurfFrame {
  T Xp[3];
  T a[3], d[3], m[3], r, v[3], h, w[3], rho, e[3], g[3], t, ca, sa;   // the quantities the derivatives reuse
  T u1[3], u3[3], lr, b1[3], b2[3];                                     // axis frames (cylinder; cone)
};

template <class T, int TY>
__device__ __forceinline__ void surf_frame(const T* G, const T* X, SurfFrame<T>& s) {
  if (TY == 0) {
#pragma unroll
    for (int i = 0; i < 3; ++i) { s.a[i] = G[i]; s.v[i] = X[i] - G[i]; }
    s.r = G[3];
    s.rho = sqrt_t(dot3(s.v, s.v));
    const T ir = T(1) / s.rho;
#pragma unroll
    for (int i = 0; i < 3; ++i) { s.e[i] = s.v[i] * ir; s.Xp[i] = s.a[i] + s.r * s.e[i]; }
  } else if (TY == 1) {
#pragma unroll
    for (int i = 0; i < 3; ++i) { s.d[i] = G[i]; s.m[i] = G[3 + i]; }
    s.r = G[6];
    cross3(s.d, s.m, s.a);   // foot p0
#pragma unroll
    for (int i = 0; i < 3; ++i) s.v[i] = X[i] - s.a[i];
    s.h = dot3(s.v, s.d);
#pragma unroll
    for (int i = 0; i < 3; ++i) s.w[i] = s.v[i] - s.h * s.d[i];
    s.rho = sqrt_t(dot3(s.w, s.w));
    const T ir = T(1) / s.rho;
#pragma unroll
    for (int i = 0; i < 3; ++i) { s.e[i] = s.w[i] * ir; s.Xp[i] = s.a[i] + s.h * s.d[i] + s.r * s.e[i]; }
    line_frame(s.d, s.m, s.u1, s.u3, s.lr);
  } else {
#pragma unroll
    for (int i = 0; i < 3; ++i) { s.a[i] = G[i]; s.d[i] = G[3 + i]; s.v[i] = X[i] - G[i]; }
    s.ca = cos((double)G[6]); s.sa = sin((double)G[6]);
    s.h = dot3(s.v, s.d);
#pragma unroll
    for (int i = 0; i < 3; ++i) s.w[i] = s.v[i] - s.h * s.d[i];
    s.rho = sqrt_t(dot3(s.w, s.w));
    const T ir = T(1) / s.rho;
#pragma unroll
    for (int i = 0; i < 3; ++i) { s.e[i] = s.w[i] * ir; s.g[i] = s.ca * s.d[i] + s.sa * s.e[i]; }
    s.t = dot3(s.v, s.g);
#pragma unroll
    for (int i = 0; i < 3; ++i) s.Xp[i] = s.a[i] + s.t * s.g[i];
    tangent_b1(s.d, s.b1);
    cross3(s.d, s.b1, s.b2);
  }
}

// dXp for a change dX of the point (grp = -1) or along group increment grp (dX ignored)
template <class T, int TY>
__device__ __forceinline__ void surf_dir(const SurfFrame<T>& s, const T* dX, int grp, T* o) {
  if (TY == 0) {
    // Xp = c + r e: de = (du - e (e.du)) / |u|, du = dX - dc
    T du[3] = {T(0), T(0), T(0)}, dc[3] = {T(0), T(0), T(0)}, ds = 0;
    if (grp < 0) { du[0] = dX[0]; du[1] = dX[1]; du[2] = dX[2]; }
    else if (grp < 3) { dc[grp] = T(1); du[grp] = T(-1); }
    else ds = T(1);
    const T ed = dot3(s.e, du), ir = T(1) / s.rho;
#pragma unroll
    for (int i = 0; i < 3; ++i) o[i] = dc[i] + s.r * (du[i] - s.e[i] * ed) * ir + s.r * ds * s.e[i];
  } else if (TY == 1) {
    T dXv[3] = {T(0), T(0), T(0)}, zeta[3] = {T(0), T(0), T(0)}, mu[3] = {T(0), T(0), T(0)}, ds = 0;
    if (grp < 0) { dXv[0] = dX[0]; dXv[1] = dX[1]; dXv[2] = dX[2]; }
    else if (grp < 4) {
      T dd[4][3], dm[4][3];
      line_dirs(s.d, s.u1, s.u3, s.lr, dd, dm);
#pragma unroll
      for (int i = 0; i < 3; ++i) { zeta[i] = dd[grp][i]; mu[i] = dm[grp][i]; }
    } else ds = T(1);
    T dp0[3], t1[3], t2[3];
    cross3(zeta, s.m, t1);
    cross3(s.d, mu, t2);
    T dv[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) { dp0[i] = t1[i] + t2[i]; dv[i] = dXv[i] - dp0[i]; }
    const T dh = dot3(dv, s.d) + dot3(s.v, zeta);
    T dw[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) dw[i] = dv[i] - dh * s.d[i] - s.h * zeta[i];
    const T ed = dot3(s.e, dw), ir = T(1) / s.rho;
#pragma unroll
    for (int i = 0; i < 3; ++i)
      o[i] = dp0[i] + dh * s.d[i] + s.h * zeta[i] + s.r * (dw[i] - s.e[i] * ed) * ir + s.r * ds * s.e[i];
  } else {
    T dXv[3] = {T(0), T(0), T(0)}, da[3] = {T(0), T(0), T(0)}, dd[3] = {T(0), T(0), T(0)}, dal = 0;
    if (grp < 0) { dXv[0] = dX[0]; dXv[1] = dX[1]; dXv[2] = dX[2]; }
    else if (grp < 3) da[grp] = T(1);
    else if (grp == 3) { dd[0] = s.b1[0]; dd[1] = s.b1[1]; dd[2] = s.b1[2]; }
    else if (grp == 4) { dd[0] = s.b2[0]; dd[1] = s.b2[1]; dd[2] = s.b2[2]; }
    else dal = T(1);
    T dv[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) dv[i] = dXv[i] - da[i];
    const T dh = dot3(dv, s.d) + dot3(s.v, dd);
    T dw[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) dw[i] = dv[i] - dh * s.d[i] - s.h * dd[i];
    const T ed = dot3(s.e, dw), ir = T(1) / s.rho;
    T dg[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const T de = (dw[i] - s.e[i] * ed) * ir;
      dg[i] = -s.sa * dal * s.d[i] + s.ca * dd[i] + s.ca * dal * s.e[i] + s.sa * de;
    }
    const T dt = dot3(dv, s.g) + dot3(s.v, dg);
#pragma unroll
    for (int i = 0; i < 3; ++i) o[i] = da[i] + dt * s.g[i] + s.t * dg[i];
  }
}

// the group-induced point residual of a sphere (TY 0), cylinder (1) or cone (2): pi(C, X) - pi(C, Proj(X))
template <class T, bool JAC, int TY, bool INTR = false>
__device__ void res_surface_point(const Cam<T>& c, const T* X, const T* G, ResJ<T>& o) {
  SurfFrame<T> s;
  surf_frame<T, TY>(G, X, s);
  T p1[3], p2[3], x1[3], x2[3], pi1[2], pi2[2], J1[2][3], J2[2][3];
  matvec3(c.R, X, p1);
  matvec3(c.R, s.Xp, p2);
#pragma unroll
  for (int i = 0; i < 3; ++i) { x1[i] = p1[i] + c.t[i]; x2[i] = p2[i] + c.t[i]; }
  o.valid = x1[2] > T(1e-6) && x2[2] > T(1e-6);
  if (!o.valid) return;
  project_dist<T, JAC>(c, x1, pi1, J1);
  project_dist<T, JAC>(c, x2, pi2, J2);
  o.r[0] = pi1[0] - pi2[0];
  o.r[1] = pi1[1] - pi2[1];
  if (!JAC) return;
  constexpr int ND = srf_dims(TY);
  T g1[2][3], g2[2][3];   // d pi / d X in world coordinates
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    T a6[6], b6[6];
    pose_row_point(p1, J1[i], a6);
    pose_row_point(p2, J2[i], b6);
#pragma unroll
    for (int k = 0; k < 6; ++k) o.Jc[i][k] = a6[k] - b6[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      g1[i][k] = J1[i][0] * c.R[k] + J1[i][1] * c.R[3 + k] + J1[i][2] * c.R[6 + k];
      g2[i][k] = J2[i][0] * c.R[k] + J2[i][1] * c.R[3 + k] + J2[i][2] * c.R[6 + k];
    }
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    T ek[3] = {T(0), T(0), T(0)}, dp[3];
    ek[k] = T(1);
    surf_dir<T, TY>(s, ek, -1, dp);
#pragma unroll
    for (int i = 0; i < 2; ++i) o.Jf[i][k] = g1[i][k] - dot3(g2[i], dp);
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    T dp[3] = {T(0), T(0), T(0)};
    if (k < ND) surf_dir<T, TY>(s, X, k, dp);
#pragma unroll
    for (int i = 0; i < 2; ++i) o.Jg[i][k] = k < ND ? -dot3(g2[i], dp) : T(0);
  }
  if (INTR) {
    T K1[2][3], K2[2][3];
    project_dist_k(c, x1, K1);
    project_dist_k(c, x2, K2);
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int k = 0; k < 3; ++k) o.Jk[i][k] = K1[i][k] - K2[i][k];
  }
}

// ---------------------------------------------------------------- ellipsoid, cuboid (Appendix B)
// Ellipsoid (R, c, s): local x = R^T (X - c), y = x / s, Xp = c + R (s y/|y|).  Cuboid (R, d): faces n_f . X + w_f
// = 0 with n_i = R e_i, w_i = -d_i and n_{i+3} = -R e_i, w_{i+3} = -d_{i+3}; Xp = X - dist_f n_f on the face
// nearest X.  Increments: R <- Exp(dw) R (3), then c (3) or d_0..2 (3) -- the first entity; log s (3) or
// d_3..5 (3) -- the second.  dXp for a change dX (grp < 0) or along increment grp (0..8).
template <class T>
struct BoxFrame {
  T Xp[3], R[9];
  T v[3], x[3], y[3], yn, yh[3], xp[3], s[3];   // ellipsoid
  T n[3], dist;                                   // cuboid: the nearest face
  int face;
};

template <class T, int TY>
__device__ __forceinline__ void box_frame(const T* G, const T* X, BoxFrame<T>& b) {
#pragma unroll
  for (int i = 0; i < 9; ++i) b.R[i] = G[i];
  if (TY == 3) {
#pragma unroll
    for (int i = 0; i < 3; ++i) { b.v[i] = X[i] - G[9 + i]; b.s[i] = G[12 + i]; }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      b.x[i] = b.R[i] * b.v[0] + b.R[3 + i] * b.v[1] + b.R[6 + i] * b.v[2];   // R^T v
      b.y[i] = b.x[i] / b.s[i];
    }
    b.yn = sqrt_t(dot3(b.y, b.y));
    const T iy = T(1) / b.yn;
#pragma unroll
    for (int i = 0; i < 3; ++i) { b.yh[i] = b.y[i] * iy; b.xp[i] = b.s[i] * b.yh[i]; }
    matvec3(b.R, b.xp, b.Xp);
#pragma unroll
    for (int i = 0; i < 3; ++i) b.Xp[i] += G[9 + i];
  } else {
    T best = T(0);
    b.face = 0;
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      const int i = f % 3;
      const T sg = f < 3 ? T(1) : T(-1);
      const T dist = sg * (b.R[i] * X[0] + b.R[3 + i] * X[1] + b.R[6 + i] * X[2]) - G[9 + f];
      if (f == 0 || fabs(dist) < fabs(best)) { best = dist; b.face = f; }
    }
    const int i = b.face % 3;
    const T sg = b.face < 3 ? T(1) : T(-1);
    b.n[0] = sg * b.R[i]; b.n[1] = sg * b.R[3 + i]; b.n[2] = sg * b.R[6 + i];
    b.dist = best;
#pragma unroll
    for (int k = 0; k < 3; ++k) b.Xp[k] = X[k] - best * b.n[k];
  }
}

template <class T, int TY>
__device__ __forceinline__ void box_dir(const BoxFrame<T>& b, const T* X, const T* dX, int grp, T* o) {
  if (TY == 3) {
    T dxw[3] = {T(0), T(0), T(0)};   // the change of X - c, before the rotation's
    T w[3] = {T(0), T(0), T(0)};     // rotation increment
    T dc[3] = {T(0), T(0), T(0)}, dls[3] = {T(0), T(0), T(0)};
    if (grp < 0) { dxw[0] = dX[0]; dxw[1] = dX[1]; dxw[2] = dX[2]; }
    else if (grp < 3) w[grp] = T(1);
    else if (grp < 6) { dc[grp - 3] = T(1); dxw[grp - 3] = T(-1); }
    else dls[grp - 6] = T(1);
    // dx = R^T (dX - dc) - R^T (w x v)
    T wv[3];
    cross3(w, b.v, wv);
    T dv[3] = {dxw[0] - wv[0], dxw[1] - wv[1], dxw[2] - wv[2]};
    T dx[3], dy[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      dx[i] = b.R[i] * dv[0] + b.R[3 + i] * dv[1] + b.R[6 + i] * dv[2];
      dy[i] = dx[i] / b.s[i] - b.y[i] * dls[i];
    }
    const T yd = dot3(b.yh, dy), iy = T(1) / b.yn;
    T dxp[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) dxp[i] = b.s[i] * dls[i] * b.yh[i] + b.s[i] * (dy[i] - b.yh[i] * yd) * iy;
    T Rdxp[3], Rxp[3], wR[3];
    matvec3(b.R, dxp, Rdxp);
    matvec3(b.R, b.xp, Rxp);
    cross3(w, Rxp, wR);
#pragma unroll
    for (int i = 0; i < 3; ++i) o[i] = dc[i] + wR[i] + Rdxp[i];
  } else {
    if (grp < 0) {
      const T nd = dot3(b.n, dX);
#pragma unroll
      for (int i = 0; i < 3; ++i) o[i] = dX[i] - nd * b.n[i];
    } else if (grp < 3) {
      T w[3] = {T(0), T(0), T(0)}, dn[3];
      w[grp] = T(1);
      cross3(w, b.n, dn);
      const T dd = dot3(dn, X);
#pragma unroll
      for (int i = 0; i < 3; ++i) o[i] = -dd * b.n[i] - b.dist * dn[i];
    } else {
      // offset d_j, j = grp - 3: only the nearest face's offset moves Xp (dist_f = n_f . X - d_f)
      const bool on = (grp - 3) == b.face;
#pragma unroll
      for (int i = 0; i < 3; ++i) o[i] = on ? b.n[i] : T(0);
    }
  }
}

// the group-induced point residual of an ellipsoid (TY 3) or cuboid (TY 4): pi(C, X) - pi(C, Proj(X)); Jg holds
// the first entity's 6 columns, Jg2 the second's 3
template <class T, bool JAC, int TY>
__device__ void res_box_point(const Cam<T>& c, const T* X, const T* G, ResJ<T>& o) {
  BoxFrame<T> b;
  box_frame<T, TY>(G, X, b);
  T p1[3], p2[3], x1[3], x2[3], pi1[2], pi2[2], J1[2][3], J2[2][3];
  matvec3(c.R, X, p1);
  matvec3(c.R, b.Xp, p2);
#pragma unroll
  for (int i = 0; i < 3; ++i) { x1[i] = p1[i] + c.t[i]; x2[i] = p2[i] + c.t[i]; }
  o.valid = x1[2] > T(1e-6) && x2[2] > T(1e-6);
  if (!o.valid) return;
  project_dist<T, JAC>(c, x1, pi1, J1);
  project_dist<T, JAC>(c, x2, pi2, J2);
  o.r[0] = pi1[0] - pi2[0];
  o.r[1] = pi1[1] - pi2[1];
  if (!JAC) return;
  T g1[2][3], g2[2][3];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    T a6[6], b6[6];
    pose_row_point(p1, J1[i], a6);
    pose_row_point(p2, J2[i], b6);
#pragma unroll
    for (int k = 0; k < 6; ++k) o.Jc[i][k] = a6[k] - b6[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      g1[i][k] = J1[i][0] * c.R[k] + J1[i][1] * c.R[3 + k] + J1[i][2] * c.R[6 + k];
      g2[i][k] = J2[i][0] * c.R[k] + J2[i][1] * c.R[3 + k] + J2[i][2] * c.R[6 + k];
    }
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    T ek[3] = {T(0), T(0), T(0)}, dp[3];
    ek[k] = T(1);
    box_dir<T, TY>(b, X, ek, -1, dp);
#pragma unroll
    for (int i = 0; i < 2; ++i) o.Jf[i][k] = g1[i][k] - dot3(g2[i], dp);
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    T dp[3];
    box_dir<T, TY>(b, X, X, k, dp);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const T v = -dot3(g2[i], dp);
      if (k < 6) o.Jg[i][k] = v; else o.Jg2[i][k - 6] = v;
    }
  }
}

// Lines on a cuboid (R, d): Eq. 8 onto the face nearest the line's point closest to the cuboid's centre
// c0 = sum_i R e_i (d_i - d_{i+3}) / 2 (no derivative through that choice).  Group columns: the rotation
// (dn = e_k x n) and the face's own offset (w = -d_f); Jg holds the first entity's 6 columns (rotation, d_0..2),
// Jg2 the second's 3 (d_3..5)
template <class T, bool JAC>
__device__ void res_box_line(const Cam<T>& c, const T* L, const T* G, const T* seg, ResJ<T>& o) {
  const T* R = G;   // row-major: column i is (R[i], R[3 + i], R[6 + i])
  const T* d = L;
  const T* m = L + 3;
  T c0[3], h[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) h[i] = T(0.5) * (G[9 + i] - G[12 + i]);
#pragma unroll
  for (int r = 0; r < 3; ++r) c0[r] = R[3 * r] * h[0] + R[3 * r + 1] * h[1] + R[3 * r + 2] * h[2];
  const T idd = T(1) / dot3(d, d);
  T p0[3], pc[3];
  cross3(d, m, p0);
#pragma unroll
  for (int i = 0; i < 3; ++i) p0[i] *= idd;
  T v[3] = {c0[0] - p0[0], c0[1] - p0[1], c0[2] - p0[2]};
  const T s = dot3(v, d) * idd;
#pragma unroll
  for (int i = 0; i < 3; ++i) pc[i] = p0[i] + s * d[i];
  T best = T(0);
  int face = 0;
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    const int i = f % 3;
    const T sg = f < 3 ? T(1) : T(-1);
    const T dist = sg * (R[i] * pc[0] + R[3 + i] * pc[1] + R[6 + i] * pc[2]) - G[9 + f];
    if (f == 0 || fabs(dist) < fabs(best)) { best = dist; face = f; }
  }
  const int fi = face % 3;
  const T sg = face < 3 ? T(1) : T(-1);
  const T n[3] = {sg * R[fi], sg * R[3 + fi], sg * R[6 + fi]};
  const T w = -G[9 + face];
  if (JAC) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
      for (int k = 0; k < 6; ++k) o.Jg[i][k] = T(0);
      o.Jg2[i][0] = o.Jg2[i][1] = o.Jg2[i][2] = T(0);
    }
  }
  plane_line_core<T, JAC, false, 4>(
      c, L, n, w, seg, o,
      [&](int k, T* dn, T& dw) {
        if (k < 3) {
          T e[3] = {T(0), T(0), T(0)};
          e[k] = T(1);
          cross3(e, n, dn);
          dw = T(0);
        } else {
          dn[0] = dn[1] = dn[2] = T(0);
          dw = T(-1);
        }
      },
      [&](int i, int k, T val) {
        if (k < 3) {
          o.Jg[i][k] = val;
        } else {
#pragma unroll
          for (int q = 0; q < 3; ++q) {   // compile-time indices: the arrays stay in registers
            if (face == q) o.Jg[i][3 + q] = val;
            if (face == 3 + q) o.Jg2[i][q] = val;
          }
        }
      });
}

// 3D wireframe endpoint distance of point X to line L = (d, m), |d| = 1: X x d - m (its norm is the distance).
// Jf: the line's 4 increments (X x dd - dm); Jk: the point's (a 3-entity of A): d/dX (X x d) = -[d]x
template <class T, bool JAC>
__device__ void res_wf3d(const T* L, const T* X, ResJ<T>& o) {
  const T* d = L;
  const T* m = L + 3;
  T xd[3];
  cross3(X, d, xd);
  o.r[0] = xd[0] - m[0]; o.r[1] = xd[1] - m[1]; o.r[2] = xd[2] - m[2];
  o.valid = true;
  if (!JAC) return;
  T u1[3], u3[3], r;
  line_frame(d, m, u1, u3, r);
  T dd[4][3], dm[4][3];
  line_dirs(d, u1, u3, r, dd, dm);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    T c[3];
    cross3(X, dd[k], c);
#pragma unroll
    for (int i = 0; i < 3; ++i) o.Jf[i][k] = c[i] - dm[k][i];
  }
  // (X + e_k) x d - X x d = e_k x d
  o.Jk[0][0] = 0;     o.Jk[0][1] = d[2];  o.Jk[0][2] = -d[1];
  o.Jk[1][0] = -d[2]; o.Jk[1][1] = 0;     o.Jk[1][2] = d[0];
  o.Jk[2][0] = d[1];  o.Jk[2][1] = -d[0]; o.Jk[2][2] = 0;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 6; ++k) o.Jc[i][k] = 0;
}

// direct 3D distance of a point to the plane (n, w): n . X + w
template <class T, bool JAC>
__device__ void res_plane_point3(const T* X, const T* P, ResJ<T>& o) {
  const T* n = P;
  o.r[0] = dot3(n, X) + P[3];
  o.valid = true;
  if (!JAC) return;
  const T* b1 = P + 4;
  const T* b2 = P + 7;
#pragma unroll
  for (int k = 0; k < 3; ++k) o.Jf[0][k] = n[k];
  o.Jg[0][0] = dot3(X, b1); o.Jg[0][1] = dot3(X, b2); o.Jg[0][2] = T(1);   // n moves along b1, b2; w along 1
#pragma unroll
  for (int k = 0; k < 6; ++k) o.Jc[0][k] = 0;
}

// direct 3D distances of a line (d, m), |d| = 1, to the plane: n . d and n . (d x m) + w (its foot point)
template <class T, bool JAC>
__device__ void res_plane_line3(const T* L, const T* P, ResJ<T>& o) {
  const T* n = P;
  const T* d = L;
  const T* m = L + 3;
  T foot[3];
  cross3(d, m, foot);
  o.r[0] = dot3(n, d);
  o.r[1] = dot3(n, foot) + P[3];
  o.valid = true;
  if (!JAC) return;
  T u1[3], u3[3], r;
  line_frame(d, m, u1, u3, r);
  T ddir[4][3], mdir[4][3];
  line_dirs(d, u1, u3, r, ddir, mdir);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    T a[3], b[3];
    cross3(ddir[k], m, a);   // d foot = dd x m + d x dm
    cross3(d, mdir[k], b);
    o.Jf[0][k] = dot3(n, ddir[k]);
    o.Jf[1][k] = n[0] * (a[0] + b[0]) + n[1] * (a[1] + b[1]) + n[2] * (a[2] + b[2]);
  }
  const T* b1 = P + 4;
  const T* b2 = P + 7;
  o.Jg[0][0] = dot3(d, b1); o.Jg[0][1] = dot3(d, b2); o.Jg[0][2] = 0;
  o.Jg[1][0] = dot3(foot, b1); o.Jg[1][1] = dot3(foot, b2); o.Jg[1][2] = T(1);
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int k = 0; k < 6; ++k) o.Jc[i][k] = 0;
}

// R6: lhat . [pi_pinhole(C, X); 1], lhat = e1 x e2 scaled to |lhat_12| = 1 (Eq. 11)
template <class T, bool JAC, bool INTR = false>
__device__ void res_p2l(const Cam<T>& c, const T* X, const T* seg, ResJ<T>& o) {
  T e1[3] = {seg[0], seg[1], T(1)}, e2[3] = {seg[2], seg[3], T(1)}, lh[3];
  cross3(e1, e2, lh);
  T s = rsqrt_t(lh[0] * lh[0] + lh[1] * lh[1]);
  lh[0] *= s; lh[1] *= s; lh[2] *= s;
  T p[3], xc[3], pi[2], J[2][3];
  matvec3(c.R, X, p);
  xc[0] = p[0] + c.t[0]; xc[1] = p[1] + c.t[1]; xc[2] = p[2] + c.t[2];
  o.valid = xc[2] > T(1e-6);
  if (!o.valid) return;
  project_pin<T, JAC>(c, xc, pi, J);
  o.r[0] = lh[0] * pi[0] + lh[1] * pi[1] + lh[2];
  if (JAC) {
    T g[3] = {lh[0] * J[0][0] + lh[1] * J[1][0], lh[0] * J[0][1] + lh[1] * J[1][1], lh[0] * J[0][2] + lh[1] * J[1][2]};
    pose_row_point(p, g, o.Jc[0]);
#pragma unroll
    for (int k = 0; k < 3; ++k) o.Jf[0][k] = g[0] * c.R[k] + g[1] * c.R[3 + k] + g[2] * c.R[6 + k];
    if (INTR) {
      // pinhole pixels pp + f (u, v): d r / d f = lhat_12 . (u, v)
      const T iz = T(1) / xc[2];
      o.Jk[0][0] = (lh[0] * xc[0] + lh[1] * xc[1]) * iz; o.Jk[0][1] = 0; o.Jk[0][2] = 0;
    }
  }
}

// R7: (l . [x;1]) / |l_12| with l = pi_l(C, L) (Eq. 12)
template <class T, bool JAC, bool INTR = false>
__device__ void res_l2p(const Cam<T>& c, const T* L, const T* x, ResJ<T>& o) {
  T dc[3], Rm[3], mc[3], l[3];
  line_to_cam(c, L, L + 3, dc, Rm, mc);
  image_line(c, mc, l);
  T A2 = l[0] * l[0] + l[1] * l[1];
  o.valid = A2 > T(1e-24);
  if (!o.valid) return;
  T in = rsqrt_t(A2);
  T q = l[0] * x[0] + l[1] * x[1] + l[2];
  o.r[0] = q * in;
  if (!JAC) return;
  // d r / d l = [x0, x1, 1]/n - q (l0, l1, 0)/n^3, then G = (d r / d l) K_l
  T in3 = in * in * in;
  T h0 = x[0] * in - q * l[0] * in3, h1 = x[1] * in - q * l[1] * in3, h2 = in;
  T G[3] = {h0 - c.px * h2, h1 - c.py * h2, c.f * h2};
  pose_row_line(c, dc, Rm, G, o.Jc[0]);
  if (INTR) { o.Jk[0][0] = mc[2] * in; o.Jk[0][1] = 0; o.Jk[0][2] = 0; }   // d l_2 / d f = m_c2, d r / d l_2 = 1/|l_12|
  T u1[3], u3[3], r;
  line_frame(L, L + 3, u1, u3, r);
  T ddir[4][3], mdir[4][3];
  line_dirs(L, u1, u3, r, ddir, mdir);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    T dm[3];
    dmc_dir(c, ddir[k], mdir[k], dm);
    o.Jf[0][k] = dot3(G, dm);
  }
}

}  // namespace ba
