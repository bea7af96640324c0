// Inter-group relations (Section 3.2, "Inter-Group Relations"; Appendix C, Manhattan / Atlanta world).
//
// A relation ties two group directions -- plane normals and VP directions -- by orthogonality (residual
// a . b, the cosine of their angle) or parallelism (residual a x b, the sine as a vector, the form of the VP
// residual).  The relations involve only kept-set parameters, so they leave the feature blocks and the
// elimination untouched: they add J^T w J to the two groups' diagonal blocks of S and to the block that
// couples them (H_gg), J^T w r to g_g, their angular Cauchy cost to E (not to the pixel cost E_px), and their
// share to the predicted decrease.  There are few of them (a handful per group), so every kernel here is a
// plain thread-per-item pass in FP64 with sums in a fixed order.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <string>
#include <vector>

#include "ba_internal.cuh"

namespace ba {

constexpr int REL_REC = 40;   // per relation: r (3), J_a (3 x 6), J_b (3 x 6), IRLS weight

static ba_status rfail(Problem& P, ba_status s, const std::string& m) {
  P.err = m;
  return s;
}
#define RCU(x)                                                              \
  do {                                                                      \
    cudaError_t e_ = (x);                                                   \
    if (e_ != cudaSuccess) {                                                \
      cudaGetLastError();                                                   \
      return rfail(P, BA_ERR_CUDA, std::string("CUDA: ") + cudaGetErrorString(e_)); \
    }                                                                       \
  } while (0)

static ba_status upload(Problem& P, int32_t*& dst, const std::vector<int32_t>& v) {
  dst = P.dnew<int32_t>((int64_t)v.size());
  if (!dst) return rfail(P, BA_ERR_OOM, "device allocation failed");
  if (!v.empty()) RCU(cudaMemcpyAsync(dst, v.data(), sizeof(int32_t) * v.size(), cudaMemcpyHostToDevice, P.stream));
  return BA_OK;
}

// Validation and the device lists (before the block pattern of S is built: the pattern takes every pair)
ba_status build_relations(Problem& P) {
  const Dims& d = P.d;
  const int64_t n = (int64_t)P.h_rel.size() / 5;
  P.nrel = n;
  if (n == 0) return BA_OK;
  const int64_t ng = d.npl + d.nv;
  std::vector<int32_t> ga(n), gb(n), ty(n);
  for (int64_t i = 0; i < n; ++i) {
    const int32_t* r = &P.h_rel[5 * i];
    auto ent = [&](int32_t kind, int32_t id, int32_t& out) -> bool {
      if (kind == BA_PLANE && id >= 0 && id < d.npl) { out = (int32_t)(d.nc + id); return true; }
      if (kind == BA_VP && id >= 0 && id < d.nv) { out = (int32_t)(d.nc + d.npl + id); return true; }
      return false;
    };
    if (!ent(r[0], r[1], ga[i]) || !ent(r[2], r[3], gb[i]))
      return rfail(P, BA_ERR_ARG, "relation " + std::to_string(i) + ": unknown group kind or id out of range");
    if (ga[i] == gb[i]) return rfail(P, BA_ERR_ARG, "relation " + std::to_string(i) + ": a group with itself");
    if (r[4] != BA_REL_ORTHOGONAL && r[4] != BA_REL_PARALLEL)
      return rfail(P, BA_ERR_ARG, "relation " + std::to_string(i) + ": unknown relation type");
    ty[i] = r[4];
  }
  // per group entity: its relations in relation order (relation << 1 | side)
  std::vector<int32_t> gp(ng + 1, 0), gi(2 * n);
  for (int64_t i = 0; i < n; ++i) { ++gp[ga[i] - d.nc + 1]; ++gp[gb[i] - d.nc + 1]; }
  for (int64_t g = 0; g < ng; ++g) gp[g + 1] += gp[g];
  {
    std::vector<int32_t> fill(gp.begin(), gp.end() - 1);
    for (int64_t i = 0; i < n; ++i) {
      gi[fill[ga[i] - d.nc]++] = (int32_t)(2 * i);
      gi[fill[gb[i] - d.nc]++] = (int32_t)(2 * i + 1);
    }
  }
  // distinct pairs (lower entity first) with their relations in relation order
  std::map<std::pair<int32_t, int32_t>, std::vector<int32_t>> pairs;
  for (int64_t i = 0; i < n; ++i) pairs[{std::min(ga[i], gb[i]), std::max(ga[i], gb[i])}].push_back((int32_t)i);
  std::vector<int32_t> pp(1, 0), pidx, pab;
  for (auto& kv : pairs) {
    for (int32_t i : kv.second) pidx.push_back(i);
    pp.push_back((int32_t)pidx.size());
    pab.push_back(kv.first.first);
    pab.push_back(kv.first.second);
  }
  P.nrelpair = (int64_t)pairs.size();
  ba_status s;
  if ((s = upload(P, P.rel_ga, ga)) || (s = upload(P, P.rel_gb, gb)) || (s = upload(P, P.rel_type, ty)) ||
      (s = upload(P, P.grel_ptr, gp)) || (s = upload(P, P.grel_idx, gi)) || (s = upload(P, P.rp_ptr, pp)) ||
      (s = upload(P, P.rp_idx, pidx)) || (s = upload(P, P.rp_pos, pab)))
    return s;
  P.rel_lin = P.dnew<double>(REL_REC * n);
  P.relH = P.dnew<double>(36 * ng);
  P.relG = P.dnew<double>(6 * ng);
  if (!P.rel_lin || !P.relH || !P.relG) return rfail(P, BA_ERR_OOM, "device allocation failed");
  RCU(cudaMemsetAsync(P.relH, 0, sizeof(double) * 36 * ng, P.stream));
  RCU(cudaMemsetAsync(P.relG, 0, sizeof(double) * 6 * ng, P.stream));
  return BA_OK;
}

// the full positions of both blocks of every pair, replacing its endpoints (after the pattern is built)
__global__ void k_rel_positions(int64_t np, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ row_len,
                                const int32_t* __restrict__ col, int32_t* __restrict__ ab) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= np) return;
  const int32_t a = ab[2 * k], b = ab[2 * k + 1];
  auto find = [&](int32_t r, int32_t c) {
    int32_t lo = row_ptr[r], hi = row_ptr[r] + row_len[r] - 1;
    while (lo < hi) {
      const int32_t mid = (lo + hi) >> 1;
      if (col[mid] < c) lo = mid + 1; else hi = mid;
    }
    return lo;
  };
  const int32_t pab = find(a, b), pba = find(b, a);
  ab[2 * k] = pab;
  ab[2 * k + 1] = pba;
}

ba_status relation_positions(Problem& P) {
  if (P.nrelpair == 0) return BA_OK;
  k_rel_positions<<<(unsigned)((P.nrelpair + 127) / 128), 128, 0, P.stream>>>(P.nrelpair, P.row_ptr, P.row_len, P.col,
                                                                               P.rp_pos);
  RCU(cudaGetLastError());
  return BA_OK;
}

// ---- a group's unit direction and its derivative along the group's increments (3 x 3 for a plane: the
// tangent basis b1, b2 of the exp-map update of the normal and a zero column for the offset; 3 x 2 for a VP)
struct GDir {
  double v[3], B[3][3];
};
__device__ __forceinline__ void group_dir(const double* grpD, int64_t gidx, GDir& o) {
  const double* D = grpD + (size_t)GRP_STRIDE * gidx;   // [n | v (3), w | 0, b1 (3), b2 (3)]
  for (int k = 0; k < 3; ++k) {
    o.v[k] = D[k];
    o.B[k][0] = D[4 + k];
    o.B[k][1] = D[7 + k];
    o.B[k][2] = 0.0;
  }
}

__device__ __forceinline__ void rel_residual(const GDir& A, const GDir& Bd, int type, double r[3], double Ja[3][3],
                                             double Jb[3][3]) {
  const double* a = A.v;
  const double* b = Bd.v;
  if (type == BA_REL_ORTHOGONAL) {
    r[0] = a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
    r[1] = r[2] = 0.0;
    for (int j = 0; j < 3; ++j) {   // d(a.b) = b . da + a . db
      Ja[0][j] = b[0] * A.B[0][j] + b[1] * A.B[1][j] + b[2] * A.B[2][j];
      Jb[0][j] = a[0] * Bd.B[0][j] + a[1] * Bd.B[1][j] + a[2] * Bd.B[2][j];
      Ja[1][j] = Ja[2][j] = Jb[1][j] = Jb[2][j] = 0.0;
    }
  } else {
    r[0] = a[1] * b[2] - a[2] * b[1];
    r[1] = a[2] * b[0] - a[0] * b[2];
    r[2] = a[0] * b[1] - a[1] * b[0];
    for (int j = 0; j < 3; ++j) {   // d(a x b) = da x b + a x db
      const double da[3] = {A.B[0][j], A.B[1][j], A.B[2][j]};
      const double db[3] = {Bd.B[0][j], Bd.B[1][j], Bd.B[2][j]};
      Ja[0][j] = da[1] * b[2] - da[2] * b[1];
      Ja[1][j] = da[2] * b[0] - da[0] * b[2];
      Ja[2][j] = da[0] * b[1] - da[1] * b[0];
      Jb[0][j] = a[1] * db[2] - a[2] * db[1];
      Jb[1][j] = a[2] * db[0] - a[0] * db[2];
      Jb[2][j] = a[0] * db[1] - a[1] * db[0];
    }
  }
}

struct RelArgs {
  int64_t n, nc, ng;
  const int32_t *ga, *gb, *type, *grel_ptr, *grel_idx, *rp_ptr, *rp_idx, *rp_pos;
  const double* grpD;   // derived group data of the parameter set in question
  double *lin, *relH, *relG;
  double w, a2;         // weight and squared Cauchy scale
};

__global__ void k_rel_lin(RelArgs a) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  GDir A, Bd;
  group_dir(a.grpD, a.ga[i] - a.nc, A);
  group_dir(a.grpD, a.gb[i] - a.nc, Bd);
  double r[3], Ja[3][3], Jb[3][3];
  rel_residual(A, Bd, a.type[i], r, Ja, Jb);
  double* o = a.lin + (size_t)REL_REC * i;
  for (int k = 0; k < 3; ++k) o[k] = r[k];
  for (int k = 0; k < 3; ++k)
    for (int j = 0; j < 6; ++j) {
      o[3 + 6 * k + j] = j < 3 ? Ja[k][j] : 0.0;
      o[21 + 6 * k + j] = j < 3 ? Jb[k][j] : 0.0;
    }
  const double s = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
  o[39] = a.w / (1.0 + s / a.a2);
}

// per group entity: sum over its relations (relation order) of J^T w J and J^T w r of its own side
__global__ void k_rel_acc(RelArgs a) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= a.ng) return;
  double H[36] = {}, G[6] = {};
  for (int k = a.grel_ptr[g]; k < a.grel_ptr[g + 1]; ++k) {
    const int e = a.grel_idx[k];
    const double* o = a.lin + (size_t)REL_REC * (e >> 1);
    const double* J = o + ((e & 1) ? 21 : 3);
    const double w = o[39];
    for (int i = 0; i < 6; ++i) {
      for (int j = 0; j < 6; ++j) H[6 * i + j] += w * (J[i] * J[j] + J[6 + i] * J[6 + j] + J[12 + i] * J[12 + j]);
      G[i] += w * (J[i] * o[0] + J[6 + i] * o[1] + J[12 + i] * o[2]);
    }
  }
  for (int k = 0; k < 36; ++k) a.relH[36 * g + k] = H[k];
  for (int k = 0; k < 6; ++k) a.relG[6 * g + k] = G[k];
}

void launch_rel_linearize(Problem& P) {
  if (!P.nrel) return;
  const Dims& d = P.d;
  RelArgs a{P.nrel, d.nc, d.npl + d.nv, P.rel_ga, P.rel_gb, P.rel_type, P.grel_ptr, P.grel_idx, P.rp_ptr,
            P.rp_idx, P.rp_pos, P.ps[P.cur].grpD, P.rel_lin, P.relH, P.relG, P.opt.w_rel,
            P.opt.cauchy_rel * P.opt.cauchy_rel};
  P.launches += 2;
  k_rel_lin<<<(unsigned)((P.nrel + 127) / 128), 128, 0, P.stream>>>(a);
  k_rel_acc<<<(unsigned)((a.ng + 127) / 128), 128, 0, P.stream>>>(a);
}

// the coupling block J_first^T w J_second of every pair, and its transpose, added to S (after the Schur pass)
template <class T>
__global__ void k_rel_offdiag(RelArgs a, int64_t npair, T* Sval, SView sv) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= npair) return;
  double C[36] = {};
  const int32_t p_ab = a.rp_pos[2 * k], p_ba = a.rp_pos[2 * k + 1];
  for (int q = a.rp_ptr[k]; q < a.rp_ptr[k + 1]; ++q) {
    const int i = a.rp_idx[q];
    const double* o = a.lin + (size_t)REL_REC * i;
    // the pair's first entity is the lower one: side a of the relation when ga < gb
    const bool a_first = a.ga[i] < a.gb[i];
    const double* J1 = o + (a_first ? 3 : 21);
    const double* J2 = o + (a_first ? 21 : 3);
    const double w = o[39];
    for (int r = 0; r < 6; ++r)
      for (int c = 0; c < 6; ++c) C[6 * r + c] += w * (J1[r] * J2[c] + J1[6 + r] * J2[6 + c] + J1[12 + r] * J2[12 + c]);
  }
  const BlkTarget t1 = sview_target(sv, p_ab), t2 = sview_target(sv, p_ba);
  for (int r = 0; r < 6; ++r)
    for (int c = 0; c < 6; ++c) {
      if (c < t1.w) Sval[t1.off + r * t1.w + c] = (T)((double)Sval[t1.off + r * t1.w + c] + C[6 * r + c]);
      if (r < t2.w) Sval[t2.off + c * t2.w + r] = (T)((double)Sval[t2.off + c * t2.w + r] + C[6 * r + c]);
    }
}

template <class T>
void launch_rel_offdiag(Problem& P) {
  if (!P.nrelpair) return;
  const Dims& d = P.d;
  RelArgs a{P.nrel, d.nc, d.npl + d.nv, P.rel_ga, P.rel_gb, P.rel_type, P.grel_ptr, P.grel_idx, P.rp_ptr,
            P.rp_idx, P.rp_pos, P.ps[P.cur].grpD, P.rel_lin, P.relH, P.relG, P.opt.w_rel,
            P.opt.cauchy_rel * P.opt.cauchy_rel};
  ++P.launches;
  k_rel_offdiag<T><<<(unsigned)((P.nrelpair + 127) / 128), 128, 0, P.stream>>>(a, P.nrelpair, (T*)P.Sval, sview_of(P));
}
template void launch_rel_offdiag<float>(Problem&);
template void launch_rel_offdiag<double>(Problem&);

// ---- cost and predicted decrease: one CTA, a fixed reduction tree
constexpr int RT = 256;
__device__ __forceinline__ double block_sum(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = RT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  const double t = sh[0];
  __syncthreads();
  return t;
}

__global__ void __launch_bounds__(RT) k_rel_cost(RelArgs a, DevScalars* S, int candidate) {
  __shared__ double sh[RT];
  double e = 0;
  for (int64_t i = threadIdx.x; i < a.n; i += RT) {
    GDir A, Bd;
    group_dir(a.grpD, a.ga[i] - a.nc, A);
    group_dir(a.grpD, a.gb[i] - a.nc, Bd);
    double r[3], Ja[3][3], Jb[3][3];
    rel_residual(A, Bd, a.type[i], r, Ja, Jb);
    const double s = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    e += 0.5 * a.w * a.a2 * log1p(s / a.a2);
  }
  const double t = block_sum(e, sh);
  if (threadIdx.x == 0) {
    if (candidate) S->Enew += t; else S->E += t;
  }
}

void launch_rel_cost(Problem& P, bool candidate) {
  if (!P.nrel) return;
  const Dims& d = P.d;
  RelArgs a{P.nrel, d.nc, d.npl + d.nv, P.rel_ga, P.rel_gb, P.rel_type, P.grel_ptr, P.grel_idx, P.rp_ptr,
            P.rp_idx, P.rp_pos, P.ps[candidate ? P.cur ^ 1 : P.cur].grpD, P.rel_lin, P.relH, P.relG,
            P.opt.w_rel, P.opt.cauchy_rel * P.opt.cauchy_rel};
  ++P.launches;
  k_rel_cost<<<1, RT, 0, P.stream>>>(a, P.S, candidate ? 1 : 0);
}

// g_rel . delta_g and sum_rel w |J_a delta_a + J_b delta_b|^2 added to the feature and camera terms
__global__ void __launch_bounds__(RT) k_rel_pred(RelArgs a, const double* __restrict__ x, DevScalars* S) {
  __shared__ double sh[RT];
  double g = 0, h = 0;
  for (int64_t k = threadIdx.x; k < a.ng; k += RT)
    for (int i = 0; i < 6; ++i) g += a.relG[6 * k + i] * x[6 * (a.nc + k) + i];
  for (int64_t i = threadIdx.x; i < a.n; i += RT) {
    const double* o = a.lin + (size_t)REL_REC * i;
    const double* xa = x + 6 * (size_t)a.ga[i];
    const double* xb = x + 6 * (size_t)a.gb[i];
    double q = 0;
    for (int k = 0; k < 3; ++k) {
      double v = 0;
      for (int j = 0; j < 6; ++j) v += o[3 + 6 * k + j] * xa[j] + o[21 + 6 * k + j] * xb[j];
      q += v * v;
    }
    h += o[39] * q;
  }
  const double tg = block_sum(g, sh);
  const double th = block_sum(h, sh);
  if (threadIdx.x == 0) {
    S->gTd += tg;
    S->dHd += th;
    S->pred = -S->gTd - 0.5 * S->dHd;
  }
}

void launch_rel_pred(Problem& P) {
  if (!P.nrel) return;
  const Dims& d = P.d;
  RelArgs a{P.nrel, d.nc, d.npl + d.nv, P.rel_ga, P.rel_gb, P.rel_type, P.grel_ptr, P.grel_idx, P.rp_ptr,
            P.rp_idx, P.rp_pos, P.ps[P.cur].grpD, P.rel_lin, P.relH, P.relG, P.opt.w_rel,
            P.opt.cauchy_rel * P.opt.cauchy_rel};
  ++P.launches;
  k_rel_pred<<<1, RT, 0, P.stream>>>(a, P.x, P.S);
}

}  // namespace ba
