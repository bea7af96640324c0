// Learned correction of the block-Jacobi preconditioner (inference and training kernels).
//
// Per diagonal block b of S (6 wide, entity = camera / plane / VP):
//   features  D_b = diag(S_bb); S^_bb = D_b^-1/2 S_bb D_b^-1/2 (21 upper entries); over the off-diagonal
//             blocks c of the row, n_bc = || D_b^-1/2 S_bc D_c^-1/2 ||_F: log(1 + count), sum, max, sum of
//             squares; entity type one-hot; zero padding to 32.
//   network   y = W2^T relu(W1^T ((x - mu) / sigma) + b1) + b2 (32 -> 128 -> 21), BF16 weights at
//             inference, FP32 accumulation.
//   block     M^ = inv(S^_bb) + sym(y) (no correction in padded / held dimensions), M = D^-1/2 M^ D^-1/2;
//             if Cholesky of M fails the block falls back to inv(S_bb) (plain block-Jacobi).
// Training (FP32, on the GPU): loss = mean_b || sym(y_b) - E_b ||_F^2 over real dimensions with
// E_b = T^_b - inv(S^_bb), T^_b the Jacobi-scaled diagonal block of the exact inverse of S.  Gradients
// are formed per CTA over a fixed slice of samples with one thread per parameter and summed over CTAs in
// order (deterministic); Adam (Kingma & Ba 2015) updates the parameters.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "ba_internal.cuh"

namespace ba {

constexpr int NF = 32, NH = 128, NO = 21;
constexpr int NPAR = 2 * NF + NF * NH + NH + NH * NO + NO;   // mu, sigma, W1, b1, W2, b2
constexpr int OFF_MU = 0, OFF_SG = NF, OFF_W1 = 2 * NF, OFF_B1 = OFF_W1 + NF * NH, OFF_W2 = OFF_B1 + NH,
              OFF_B2 = OFF_W2 + NH * NO;
constexpr int NTRAIN = NPAR - 2 * NF;

__device__ __constant__ int c_iu[21] = {0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 2, 2, 2, 2, 3, 3, 3, 4, 4, 5};
__device__ __constant__ int c_ju[21] = {0, 1, 2, 3, 4, 5, 1, 2, 3, 4, 5, 2, 3, 4, 5, 3, 4, 5, 4, 5, 5};

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// real (non-padding, non-held) dimensions of entity a as a 6-bit mask
__device__ __forceinline__ unsigned real_mask(int64_t a, int64_t nc, const uint8_t* ent_type, const uint8_t* held) {
  const int nd = ent_dims(ent_type[a]);
  unsigned m = (1u << nd) - 1u;
  if (a < nc) m &= ~(unsigned)held[a];
  return m;
}

// ---------------------------------------------------------------- features (warp per block row)
template <class T>
__global__ void k_pre_features(int64_t na, int64_t nc, const int32_t* __restrict__ row_ptr,
                               const int32_t* __restrict__ row_len, const int32_t* __restrict__ col,
                               const T* __restrict__ Sval, const double* __restrict__ sdiag,
                               const uint8_t* __restrict__ ent_type, const uint8_t* __restrict__ held,
                               float* __restrict__ X, uint8_t* __restrict__ mask, SView sv) {
  const int lane = threadIdx.x & 31;
  const int64_t a = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (a >= na) return;
  double sda[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) sda[i] = 1.0 / sqrt(fmax(sdiag[6 * a + i], 1e-300));
  double cnt = 0, s1 = 0, mx = 0, s2 = 0;
  const int q0 = row_ptr[a], q1 = q0 + row_len[a];
  for (int q = q0 + lane; q < q1; q += 32) {
    const int c = col[q];
    double blk[36];
    sview_load(sv, Sval, q, a, blk);
    if (c == a) {
      for (int k = 0; k < NO; ++k) {
        const int i = c_iu[k], j = c_ju[k];
        X[(size_t)a * NF + k] = (float)(sda[i] * blk[i * 6 + j] * sda[j]);
      }
    } else {
      double sdc[6];
#pragma unroll
      for (int j = 0; j < 6; ++j) sdc[j] = 1.0 / sqrt(fmax(sdiag[6 * (size_t)c + j], 1e-300));
      double f2 = 0;
#pragma unroll
      for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = 0; j < 6; ++j) {
          const double v = sda[i] * blk[i * 6 + j] * sdc[j];
          f2 += v * v;
        }
      const double n = sqrt(f2);
      cnt += 1; s1 += n; s2 += f2; mx = fmax(mx, n);
    }
  }
  cnt = warp_sum_d(cnt); s1 = warp_sum_d(s1); s2 = warp_sum_d(s2); mx = warp_max_d(mx);
  if (lane == 0) {
    float* x = X + (size_t)a * NF;
    x[21] = (float)log1p(cnt); x[22] = (float)s1; x[23] = (float)mx; x[24] = (float)s2;
    const int et = ent_type[a];
    x[25] = et == 0; x[26] = et == 1 || et == 3; x[27] = et == 2;   // an intrinsics block counts as a 3-wide group
    x[28] = x[29] = x[30] = x[31] = 0.f;
    mask[a] = (uint8_t)real_mask(a, nc, ent_type, held);
  }
}

// ---------------------------------------------------------------- inference (thread per block row)
__device__ bool chol_inv6(const double (&A)[6][6], double (&Ai)[6][6]) {
  double L[6][6] = {};
  for (int j = 0; j < 6; ++j) {
    double s = A[j][j];
    for (int k = 0; k < j; ++k) s -= L[j][k] * L[j][k];
    if (!(s > 0)) return false;
    L[j][j] = sqrt(s);
    for (int i = j + 1; i < 6; ++i) {
      double t = A[i][j];
      for (int k = 0; k < j; ++k) t -= L[i][k] * L[j][k];
      L[i][j] = t / L[j][j];
    }
  }
  double Li[6][6] = {};
  for (int i = 0; i < 6; ++i) {
    Li[i][i] = 1.0 / L[i][i];
    for (int j = 0; j < i; ++j) {
      double s = 0;
      for (int k = j; k < i; ++k) s += L[i][k] * Li[k][j];
      Li[i][j] = -s * Li[i][i];
    }
  }
  for (int i = 0; i < 6; ++i)
    for (int j = i; j < 6; ++j) {
      double s = 0;
      for (int k = j; k < 6; ++k) s += Li[k][i] * Li[k][j];
      Ai[i][j] = s; Ai[j][i] = s;
    }
  return true;
}

template <class T>
__global__ void __launch_bounds__(128) k_pre_learned(int64_t na, const int32_t* __restrict__ row_ptr,
                                                    const int32_t* __restrict__ row_len, const int32_t* __restrict__ col,
                                                    const T* __restrict__ Sval, const double* __restrict__ sdiag,
                                                    const float* __restrict__ X, const uint8_t* __restrict__ mask,
                                                    const float* __restrict__ prm, const __nv_bfloat16* __restrict__ w1h,
                                                    const __nv_bfloat16* __restrict__ w2h, T* __restrict__ Minv,
                                                    int* __restrict__ fallbacks, SView sv) {
  __shared__ __nv_bfloat16 sW1[NF * NH];
  __shared__ __nv_bfloat16 sW2[NH * NO];
  __shared__ float sB1[NH], sB2[NO], sMu[NF], sSg[NF];
  for (int i = threadIdx.x; i < NF * NH; i += blockDim.x) sW1[i] = w1h[i];
  for (int i = threadIdx.x; i < NH * NO; i += blockDim.x) sW2[i] = w2h[i];
  for (int i = threadIdx.x; i < NH; i += blockDim.x) sB1[i] = prm[OFF_B1 + i];
  for (int i = threadIdx.x; i < NO; i += blockDim.x) sB2[i] = prm[OFF_B2 + i];
  for (int i = threadIdx.x; i < NF; i += blockDim.x) { sMu[i] = prm[OFF_MU + i]; sSg[i] = prm[OFF_SG + i]; }
  __syncthreads();
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= na) return;
  // network
  float z[NF];
#pragma unroll
  for (int i = 0; i < NF; ++i) z[i] = (X[(size_t)a * NF + i] - sMu[i]) / sSg[i];
  float y[NO];
#pragma unroll
  for (int o = 0; o < NO; ++o) y[o] = sB2[o];
  for (int k = 0; k < NH; ++k) {
    float h = sB1[k];
#pragma unroll
    for (int i = 0; i < NF; ++i) h = fmaf(z[i], __bfloat162float(sW1[i * NH + k]), h);
    h = fmaxf(h, 0.f);
#pragma unroll
    for (int o = 0; o < NO; ++o) y[o] = fmaf(h, __bfloat162float(sW2[k * NO + o]), y[o]);
  }
  // the diagonal block and its scaled inverse
  int pos = row_ptr[a];
  for (int q = row_ptr[a]; q < row_ptr[a] + row_len[a]; ++q)
    if (col[q] == a) { pos = q; break; }
  double sd[6], Sh[6][6], Shi[6][6];
  bool pos_diag = true;
  for (int i = 0; i < 6; ++i) {
    pos_diag &= sdiag[6 * a + i] > 0;
    sd[i] = 1.0 / sqrt(fmax(sdiag[6 * a + i], 1e-300));
  }
  const int64_t dof = sview_target(sv, pos).off;   // the diagonal block is stored whole
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) Sh[i][j] = sd[i] * (double)Sval[dof + i * 6 + j] * sd[j];
  // symmetric part (the stored diagonal block is symmetric already)
  bool ok = pos_diag && chol_inv6(Sh, Shi);
  const unsigned m = mask[a];
  double M[6][6];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) M[i][j] = Shi[i][j];
  if (ok) {
    for (int k = 0; k < NO; ++k) {
      const int i = c_iu[k], j = c_ju[k];
      if (((m >> i) & 1u) && ((m >> j) & 1u)) {
        M[i][j] += y[k];
        if (i != j) M[j][i] += y[k];
      }
    }
    double Mu[6][6], tmp[6][6];
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j) Mu[i][j] = sd[i] * M[i][j] * sd[j];
    // positive-definiteness check of the corrected block (its inverse is not needed)
    if (!chol_inv6(Mu, tmp)) {
      atomicAdd(fallbacks, 1);
      for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) Mu[i][j] = sd[i] * Shi[i][j] * sd[j];
    }
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j) Minv[(size_t)a * BS2 + i * 6 + j] = (T)Mu[i][j];
  } else {
    atomicAdd(fallbacks, 1);
    // the diagonal block itself is not positive definite: the same diagonal fall-back as block-Jacobi
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j)
        Minv[(size_t)a * BS2 + i * 6 + j] =
            (T)(i == j ? (sdiag[6 * a + i] > 0 ? 1.0 / sdiag[6 * a + i] : 1.0) : 0.0);
  }
}

__global__ void k_to_bf16(int n, const float* __restrict__ a, __nv_bfloat16* __restrict__ b) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = __float2bfloat16(a[i]);
}

// ---------------------------------------------------------------- training
constexpr int TB = 64;     // samples per CTA slice
constexpr int TT = 256;    // threads per CTA

// per-CTA partial gradient of the trained parameters over samples [s0, s0 + TB) of [0, n)
__global__ void __launch_bounds__(TT) k_mlp_grad_part(int64_t n, int64_t off, int64_t total, double inv_count,
                                                      const float* __restrict__ X, const float* __restrict__ E,
                                                      const uint8_t* __restrict__ mask, const float* __restrict__ prm,
                                                      float* __restrict__ gpart, double* __restrict__ lpart) {
  extern __shared__ float sm[];
  float* sZ = sm;                       // TB x NF
  float* sA = sZ + TB * NF;             // TB x NH (pre-activation, then dA)
  float* sH = sA + TB * NH;             // TB x NH
  float* sY = sH + TB * NH;             // TB x NO (then dY)
  float* sW1 = sY + TB * NO;            // NF x NH
  float* sW2 = sW1 + NF * NH;           // NH x NO
  __shared__ double lsh[TT / 32];
  const int64_t s0 = (int64_t)blockIdx.x * TB;
  const int ns = (int)((n - s0) < TB ? (n - s0) : TB);
  for (int i = threadIdx.x; i < NF * NH; i += TT) sW1[i] = prm[OFF_W1 + i];
  for (int i = threadIdx.x; i < NH * NO; i += TT) sW2[i] = prm[OFF_W2 + i];
  for (int i = threadIdx.x; i < TB * NF; i += TT) {
    const int s = i / NF, f = i % NF;
    const int64_t g = (off + s0 + s) % total;
    sZ[i] = s < ns ? (X[g * NF + f] - prm[OFF_MU + f]) / prm[OFF_SG + f] : 0.f;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < TB * NH; i += TT) {
    const int s = i / NH, k = i % NH;
    float acc = prm[OFF_B1 + k];
    for (int f = 0; f < NF; ++f) acc = fmaf(sZ[s * NF + f], sW1[f * NH + k], acc);
    sA[i] = acc;
    sH[i] = fmaxf(acc, 0.f);
  }
  __syncthreads();
  double lacc = 0;
  for (int i = threadIdx.x; i < TB * NO; i += TT) {
    const int s = i / NO, o = i % NO;
    float y = prm[OFF_B2 + o];
    for (int k = 0; k < NH; ++k) y = fmaf(sH[s * NH + k], sW2[k * NO + o], y);
    float dy = 0.f;
    if (s < ns) {
      const int64_t g = (off + s0 + s) % total;
      const unsigned m = mask[g];
      const int ii = c_iu[o], jj = c_ju[o];
      if (((m >> ii) & 1u) && ((m >> jj) & 1u)) {
        const float r = y - E[g * NO + o];
        const float w = ii == jj ? 1.f : 2.f;
        lacc += (double)w * r * r;
        dy = (float)(2.0 * w * r * inv_count);
      }
    }
    sY[i] = dy;
  }
  // loss partial: warp sums, then warp partials in order
  lacc = warp_sum_d(lacc);
  if ((threadIdx.x & 31) == 0) lsh[threadIdx.x >> 5] = lacc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < TT / 32; ++w) t += lsh[w];
    lpart[blockIdx.x] = t * inv_count;
  }
  // dA = (dY W2^T) * [A > 0]
  for (int i = threadIdx.x; i < TB * NH; i += TT) {
    const int s = i / NH, k = i % NH;
    float d = 0.f;
    for (int o = 0; o < NO; ++o) d = fmaf(sY[s * NO + o], sW2[k * NO + o], d);
    sA[i] = sA[i] > 0.f ? d : 0.f;
  }
  __syncthreads();
  // one thread per trained parameter, samples in order
  float* gp = gpart + (size_t)blockIdx.x * NTRAIN;
  for (int j = threadIdx.x; j < NTRAIN; j += TT) {
    float g = 0.f;
    if (j < NF * NH) {                                  // W1[f][k]
      const int f = j / NH, k = j % NH;
      for (int s = 0; s < ns; ++s) g = fmaf(sZ[s * NF + f], sA[s * NH + k], g);
    } else if (j < NF * NH + NH) {                      // b1[k]
      const int k = j - NF * NH;
      for (int s = 0; s < ns; ++s) g += sA[s * NH + k];
    } else if (j < NF * NH + NH + NH * NO) {            // W2[k][o]
      const int t = j - NF * NH - NH, k = t / NO, o = t % NO;
      for (int s = 0; s < ns; ++s) g = fmaf(sH[s * NH + k], sY[s * NO + o], g);
    } else {                                            // b2[o]
      const int o = j - NF * NH - NH - NH * NO;
      for (int s = 0; s < ns; ++s) g += sY[s * NO + o];
    }
    gp[j] = g;
  }
}

__global__ void k_mlp_grad_sum(int nblk, const float* __restrict__ gpart, const double* __restrict__ lpart,
                               float* __restrict__ grad, double* __restrict__ loss) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < NTRAIN) {
    double g = 0;
    for (int b = 0; b < nblk; ++b) g += gpart[(size_t)b * NTRAIN + j];
    grad[j] = (float)g;
  }
  if (j == 0 && loss) {
    double l = 0;
    for (int b = 0; b < nblk; ++b) l += lpart[b];
    *loss = l;
  }
}

__global__ void k_adam(float* __restrict__ prm, float* __restrict__ m, float* __restrict__ v, const float* __restrict__ g,
                       int t, float lr, float b1, float b2, float eps) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= NTRAIN) return;
  const float gj = g[j];
  const float mj = b1 * m[j] + (1.f - b1) * gj;
  const float vj = b2 * v[j] + (1.f - b2) * gj * gj;
  m[j] = mj;
  v[j] = vj;
  const float mh = mj / (1.f - powf(b1, (float)t));
  const float vh = vj / (1.f - powf(b2, (float)t));
  prm[2 * NF + j] -= lr * mh / (sqrtf(vh) + eps);
}

static size_t grad_smem() { return sizeof(float) * (TB * NF + 2 * TB * NH + TB * NO + NF * NH + NH * NO); }

// gradient of the loss over samples [off, off + n) (wrapping modulo total), normalised by n
static cudaError_t mlp_grad(cudaStream_t st, int64_t off, int64_t n, int64_t total, const float* X, const float* E,
                            const uint8_t* mask, const float* prm, float* gpart, double* lpart, float* grad,
                            double* loss) {
  const int nblk = (int)((n + TB - 1) / TB);
  cudaFuncSetAttribute(k_mlp_grad_part, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)grad_smem());
  k_mlp_grad_part<<<nblk, TT, grad_smem(), st>>>(n, off, total, 1.0 / (double)n, X, E, mask, prm, gpart, lpart);
  k_mlp_grad_sum<<<(NTRAIN + 255) / 256, 256, 0, st>>>(nblk, gpart, lpart, grad, loss);
  return cudaGetLastError();
}

}  // namespace ba

using namespace ba;

// ---------------------------------------------------------------- C ABI
extern "C" int ba_precond_param_count(void) { return NPAR; }

// work buffer (floats): per-CTA partial gradients, then (8-byte aligned) per-CTA loss partials, the loss,
// then the gradient
static int64_t work_a(int64_t nblk) { return ((nblk * NTRAIN + 1) / 2) * 2; }

extern "C" int64_t ba_mlp_work_floats(int64_t batch) {
  const int64_t nblk = (batch + TB - 1) / TB;
  return work_a(nblk) + 2 * nblk + 2 + NTRAIN;
}

extern "C" ba_status ba_mlp_grad(int64_t n, const float* X, const float* E, const uint8_t* mask, const float* params,
                                 float* grad, double* loss, float* work, void* cuda_stream) {
  if (n <= 0 || !X || !E || !mask || !params || !grad || !work) return BA_ERR_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int64_t nblk = (n + TB - 1) / TB;
  float* gpart = work;
  double* lpart = (double*)(work + work_a(nblk));
  double* dloss = lpart + nblk;
  cudaError_t e = mlp_grad(st, 0, n, n, X, E, mask, params, gpart, lpart, grad, dloss);
  if (e != cudaSuccess) return BA_ERR_CUDA;
  if (loss && cudaMemcpyAsync(loss, dloss, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess) return BA_ERR_CUDA;
  return cudaStreamSynchronize(st) == cudaSuccess ? BA_OK : BA_ERR_CUDA;
}

extern "C" ba_status ba_precond_train(int64_t n, const float* X, const float* E, const uint8_t* mask, float* params,
                                      float* adam_m, float* adam_v, int t0, int steps, int64_t batch, float lr,
                                      float* work, double* loss_last, void* cuda_stream) {
  if (n <= 0 || batch <= 0 || steps < 0 || t0 < 0 || !X || !E || !mask || !params || !adam_m || !adam_v || !work)
    return BA_ERR_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int64_t b = batch < n ? batch : n;
  const int64_t nblk = (b + TB - 1) / TB;
  float* gpart = work;
  double* lpart = (double*)(work + work_a(nblk));
  double* dloss = lpart + nblk;
  float* grad = (float*)(dloss + 1);
  for (int s = 0; s < steps; ++s) {
    const int64_t off = ((int64_t)s * b) % n;
    cudaError_t e = mlp_grad(st, off, b, n, X, E, mask, params, gpart, lpart, grad, dloss);
    if (e != cudaSuccess) return BA_ERR_CUDA;
    k_adam<<<(NTRAIN + 255) / 256, 256, 0, st>>>(params, adam_m, adam_v, grad, t0 + s + 1, lr, 0.9f, 0.999f, 1e-8f);
  }
  if (cudaGetLastError() != cudaSuccess) return BA_ERR_CUDA;
  if (loss_last && steps > 0 && cudaMemcpyAsync(loss_last, dloss, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return BA_ERR_CUDA;
  return cudaStreamSynchronize(st) == cudaSuccess ? BA_OK : BA_ERR_CUDA;
}

// ---------------------------------------------------------------- hooks used by the step (api.cu)
namespace ba {

ba_status precond_set_weights(Problem& P, const float* host_params) {
  if (!P.pre_params) {
    P.pre_params = P.dnew<float>(NPAR);
    P.pre_w1 = (void*)P.dnew<__nv_bfloat16>(NF * NH);
    P.pre_w2 = (void*)P.dnew<__nv_bfloat16>(NH * NO);
    P.pre_fallbacks = P.dnew<int>(1);
    if (!P.pre_params || !P.pre_w1 || !P.pre_w2 || !P.pre_fallbacks) return BA_ERR_OOM;
  }
  if (cudaMemcpyAsync(P.pre_params, host_params, sizeof(float) * NPAR, cudaMemcpyHostToDevice, P.stream) != cudaSuccess)
    return BA_ERR_CUDA;
  k_to_bf16<<<(NF * NH + 255) / 256, 256, 0, P.stream>>>(NF * NH, P.pre_params + OFF_W1, (__nv_bfloat16*)P.pre_w1);
  k_to_bf16<<<(NH * NO + 255) / 256, 256, 0, P.stream>>>(NH * NO, P.pre_params + OFF_W2, (__nv_bfloat16*)P.pre_w2);
  if (cudaStreamSynchronize(P.stream) != cudaSuccess) return BA_ERR_CUDA;
  P.pre_ready = true;
  return BA_OK;
}

ba_status precond_alloc_features(Problem& P) {
  if (!P.pre_X) {
    P.pre_X = P.dnew<float>(NF * P.d.na);
    P.pre_mask = P.dnew<uint8_t>(P.d.na);
    if (!P.pre_X || !P.pre_mask) return BA_ERR_OOM;
  }
  return BA_OK;
}

template <class T>
void launch_pre_features(Problem& P) {
  const Dims& d = P.d;
  ++P.launches;
  k_pre_features<T><<<(int)((d.na * 32 + 127) / 128), 128, 0, P.stream>>>(
      d.na, d.nc, P.row_ptr, P.row_len, P.col, (const T*)P.Sval, P.sdiag, P.ent_type, P.cam_fixed, P.pre_X, P.pre_mask,
      sview_of(P));
}

template <class T>
void launch_pre_learned(Problem& P) {
  const Dims& d = P.d;
  cudaMemsetAsync(P.pre_fallbacks, 0, sizeof(int), P.stream);
  launch_pre_features<T>(P);
  ++P.launches;
  k_pre_learned<T><<<(int)((d.na + 127) / 128), 128, 0, P.stream>>>(
      d.na, P.row_ptr, P.row_len, P.col, (const T*)P.Sval, P.sdiag, P.pre_X, P.pre_mask, P.pre_params,
      (const __nv_bfloat16*)P.pre_w1, (const __nv_bfloat16*)P.pre_w2, (T*)P.Minv, P.pre_fallbacks, sview_of(P));
}

template void launch_pre_features<float>(Problem&);
template void launch_pre_features<double>(Problem&);
template void launch_pre_learned<float>(Problem&);
template void launch_pre_learned<double>(Problem&);

}  // namespace ba
