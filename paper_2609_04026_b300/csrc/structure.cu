// One-time structure build (K0): the analogue of a sparse solver's symbolic
// analysis, which the paper observes only on the first iteration of each BA
// call (Section 4, Fig. 3c).  It runs on the host once per problem:
//   * validates every index (BA_ERR_ARG on failure),
//   * orders the residual records feature-major (each residual touches exactly
//     one feature, Section 3.2-3.4, so H_ff is block-diagonal),
//   * gives every (feature, kept entity) pair a "slot" that will hold its
//     W block and its direct contribution to H_aa,
//   * builds the block pattern of S over A = cameras u groups (every pair of
//     entities that share a feature, Section 3.3 sparsity analysis), stored as
//     full block-CSR (both triangles, for the SpMV),
//   * lists, for every upper block of S, the slot pairs (e_a, e_b) whose product
//     W_a V^-1 W_b^T lands in it, cut into work items of at most PAIR_CHUNK pairs
//     so that the Schur kernel accumulates each block in a fixed order without
//     atomics.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "ba_internal.cuh"

namespace ba {

static constexpr int PAIR_CHUNK = 64;

static ba_status fail(Problem& P, ba_status s, const std::string& m) {
  P.err = m;
  return s;
}

#define CU(x)                                                                   \
  do {                                                                          \
    cudaError_t e_ = (x);                                                       \
    if (e_ != cudaSuccess) return fail(P, BA_ERR_CUDA, std::string(#x ": ") + cudaGetErrorString(e_)); \
  } while (0)

template <class X>
static ba_status upload(Problem& P, X*& dst, const std::vector<X>& src) {
  dst = P.dnew<X>((int64_t)src.size());
  if (!dst) return fail(P, BA_ERR_OOM, "device allocation failed");
  if (!src.empty())
    CU(cudaMemcpyAsync(dst, src.data(), sizeof(X) * src.size(), cudaMemcpyHostToDevice, P.stream));
  return BA_OK;
}

ba_status build_structure(Problem& P) {
  Dims& d = P.d;
  d.nc = (int64_t)P.h_cam.size() / 12;
  d.np = (int64_t)P.h_pts.size() / 3;
  d.nl = (int64_t)P.h_lin.size() / 6;
  d.npl = (int64_t)P.h_pln.size() / 4;
  d.nv = (int64_t)P.h_vps.size() / 3;
  d.nf = d.np + d.nl;
  d.na = d.nc + d.npl + d.nv;
  if (d.na > (int64_t)1 << 30 || d.nf > (int64_t)1 << 30) return fail(P, BA_ERR_ARG, "too many entities");

  // ---- normalise parameters: unit quaternions, |d| = 1 lines, unit plane normals (with w), unit VPs
  for (int64_t i = 0; i < d.nc; ++i) {
    double* q = &P.h_cam[12 * i];
    double n = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    if (!(n > 0) || !std::isfinite(n)) return fail(P, BA_ERR_ARG, "camera " + std::to_string(i) + ": zero quaternion");
    for (int k = 0; k < 4; ++k) q[k] /= n;
  }
  for (int64_t i = 0; i < d.nl; ++i) {
    double* L = &P.h_lin[6 * i];
    double n = std::sqrt(L[0] * L[0] + L[1] * L[1] + L[2] * L[2]);
    if (!(n > 0) || !std::isfinite(n)) return fail(P, BA_ERR_ARG, "line " + std::to_string(i) + ": zero direction");
    for (int k = 0; k < 6; ++k) L[k] /= n;
  }
  for (int64_t i = 0; i < d.npl; ++i) {
    double* Q = &P.h_pln[4 * i];
    double n = std::sqrt(Q[0] * Q[0] + Q[1] * Q[1] + Q[2] * Q[2]);
    if (!(n > 0) || !std::isfinite(n)) return fail(P, BA_ERR_ARG, "plane " + std::to_string(i) + ": zero normal");
    for (int k = 0; k < 4; ++k) Q[k] /= n;
  }
  for (int64_t i = 0; i < d.nv; ++i) {
    double* v = &P.h_vps[3 * i];
    double n = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    if (!(n > 0) || !std::isfinite(n)) return fail(P, BA_ERR_ARG, "vp " + std::to_string(i) + ": zero direction");
    for (int k = 0; k < 3; ++k) v[k] /= n;
  }

  // ---- gather and validate residual records
  int64_t nr = 0;
  for (auto& b : P.h_obs) nr += (int64_t)b.feat.size();
  if (nr > (int64_t)INT32_MAX - 1) return fail(P, BA_ERR_ARG, "too many residuals");
  d.nr = nr;
  std::vector<int8_t> kind(nr);
  std::vector<int32_t> cam(nr), feat(nr), grp(nr);
  std::vector<double> meas(4 * nr);
  {
    int64_t o = 0;
    for (auto& b : P.h_obs) {
      int64_t n = (int64_t)b.feat.size();
      for (int64_t i = 0; i < n; ++i, ++o) {
        int k = b.kind;
        kind[o] = (int8_t)k;
        bool is_point = (k == R_POINT || k == R_PLANE_POINT || k == R_P2L);
        int32_t f = b.feat[i];
        int64_t nfk = is_point ? d.np : d.nl;
        if (f < 0 || f >= nfk) return fail(P, BA_ERR_ARG, "observation kind " + std::to_string(k) + ": feature id out of range");
        feat[o] = is_point ? f : (int32_t)(d.np + f);
        if (k != R_VP) {
          int32_t c = b.cam[i];
          if (c < 0 || c >= d.nc) return fail(P, BA_ERR_ARG, "observation kind " + std::to_string(k) + ": camera id out of range");
          cam[o] = c;
        } else {
          cam[o] = -1;
        }
        grp[o] = -1;
        if (k == R_PLANE_POINT || k == R_PLANE_LINE) {
          int32_t g = b.other[i];
          if (g < 0 || g >= d.npl) return fail(P, BA_ERR_ARG, "plane id out of range");
          grp[o] = g;
        } else if (k == R_VP) {
          int32_t g = b.other[i];
          if (g < 0 || g >= d.nv) return fail(P, BA_ERR_ARG, "vp id out of range");
          grp[o] = g;
        } else if (k == R_P2L || k == R_L2P) {
          if (!b.other.empty()) {
            int32_t g = b.other[i];
            int64_t lim = (k == R_P2L) ? d.nl : d.np;
            if (g < 0 || g >= lim) return fail(P, BA_ERR_ARG, "partner feature id out of range");
          }
        }
        for (int c = 0; c < 4; ++c) meas[4 * o + c] = b.meas[4 * i + c];
      }
    }
  }
  P.h_obs.clear();
  P.h_obs.shrink_to_fit();

  // ---- feature-major order (counting sort by feature, then by camera inside a feature)
  std::vector<int32_t> fres_off(d.nf + 1, 0);
  for (int64_t i = 0; i < nr; ++i) fres_off[feat[i] + 1]++;
  for (int64_t f = 0; f < d.nf; ++f) fres_off[f + 1] += fres_off[f];
  std::vector<int32_t> order(nr);
  {
    std::vector<int32_t> pos(fres_off.begin(), fres_off.end() - 1);
    for (int64_t i = 0; i < nr; ++i) order[pos[feat[i]]++] = (int32_t)i;
  }
  for (int64_t f = 0; f < d.nf; ++f) {
    auto b = order.begin() + fres_off[f], e = order.begin() + fres_off[f + 1];
    std::stable_sort(b, e, [&](int32_t a, int32_t c) { return cam[a] < cam[c]; });
  }
  d.n_points_res_end = fres_off[d.np];

  // ---- slots: one per (feature, kept entity); cameras first (ids < groups)
  std::vector<int32_t> fslot_off(d.nf + 1, 0);
  std::vector<int32_t> slot_ent, slot_feat;
  std::vector<uint8_t> slot_type;
  std::vector<int32_t> feat_plane_slot(d.nf, -1);
  std::vector<int32_t> rslot_c(nr, -1), rslot_g(nr, -1);
  slot_ent.reserve((size_t)nr + d.nf);
  {
    std::vector<int32_t> ents;
    for (int64_t f = 0; f < d.nf; ++f) {
      ents.clear();
      int32_t plane = -1, vp = -1;
      for (int32_t j = fres_off[f]; j < fres_off[f + 1]; ++j) {
        int32_t i = order[j];
        if (cam[i] >= 0 && P.h_fixed[cam[i]] != 0x3F) ents.push_back(cam[i]);
        int k = kind[i];
        if (k == R_PLANE_POINT || k == R_PLANE_LINE) {
          if (plane >= 0 && plane != grp[i]) return fail(P, BA_ERR_ARG, "a feature may be associated with at most one plane");
          plane = grp[i];
        }
        if (k == R_VP) {
          if (vp >= 0 && vp != grp[i]) return fail(P, BA_ERR_ARG, "a line may be associated with at most one VP");
          vp = grp[i];
        }
      }
      if (plane >= 0) ents.push_back((int32_t)(d.nc + plane));
      if (vp >= 0) ents.push_back((int32_t)(d.nc + d.npl + vp));
      std::sort(ents.begin(), ents.end());
      ents.erase(std::unique(ents.begin(), ents.end()), ents.end());
      int32_t base = (int32_t)slot_ent.size();
      fslot_off[f] = base;
      for (int32_t a : ents) {
        slot_ent.push_back(a);
        slot_feat.push_back((int32_t)f);
        uint8_t t = a < d.nc ? ENT_CAM : (a < d.nc + d.npl ? ENT_PLANE : ENT_VP);
        slot_type.push_back(t);
        if (t == ENT_PLANE) feat_plane_slot[f] = (int32_t)(slot_ent.size() - 1);
      }
      for (int32_t j = fres_off[f]; j < fres_off[f + 1]; ++j) {
        int32_t i = order[j];
        auto find = [&](int32_t a) {
          auto it = std::lower_bound(ents.begin(), ents.end(), a);
          return base + (int32_t)(it - ents.begin());
        };
        if (cam[i] >= 0 && P.h_fixed[cam[i]] != 0x3F) rslot_c[j] = find(cam[i]);
        int k = kind[i];
        if (k == R_PLANE_POINT || k == R_PLANE_LINE) rslot_g[j] = find((int32_t)(d.nc + grp[i]));
        if (k == R_VP) rslot_g[j] = find((int32_t)(d.nc + d.npl + grp[i]));
      }
      if ((int64_t)slot_ent.size() > INT32_MAX - 1) return fail(P, BA_ERR_ARG, "too many slots");
    }
    fslot_off[d.nf] = (int32_t)slot_ent.size();
  }
  d.ne = (int64_t)slot_ent.size();
  P.line_slot0 = fslot_off[d.np];

  // ---- upper block pattern of S: all entity pairs that share a feature, plus every diagonal
  const int64_t na = d.na;
  std::vector<int32_t> up_ptr(na + 1, 0), up_col;
  {
    std::vector<std::vector<int32_t>> rows(na);
    for (int64_t a = 0; a < na; ++a) rows[a].push_back((int32_t)a);
    for (int64_t f = 0; f < d.nf; ++f)
      for (int32_t i = fslot_off[f]; i < fslot_off[f + 1]; ++i)
        for (int32_t j = i + 1; j < fslot_off[f + 1]; ++j) rows[slot_ent[i]].push_back(slot_ent[j]);
    for (int64_t a = 0; a < na; ++a) {
      auto& r = rows[a];
      std::sort(r.begin(), r.end());
      r.erase(std::unique(r.begin(), r.end()), r.end());
      up_ptr[a + 1] = up_ptr[a] + (int32_t)r.size();
    }
    up_col.resize(up_ptr[na]);
    for (int64_t a = 0; a < na; ++a) std::copy(rows[a].begin(), rows[a].end(), up_col.begin() + up_ptr[a]);
  }
  d.nbu = up_ptr[na];
  std::vector<int32_t> up_row(d.nbu);
  for (int64_t a = 0; a < na; ++a)
    for (int32_t u = up_ptr[a]; u < up_ptr[a + 1]; ++u) up_row[u] = (int32_t)a;

  // ---- full block-CSR (row b = lower entries (cols a < b, ascending) then upper entries)
  std::vector<int32_t> row_ptr(na + 1, 0), low_cnt(na, 0);
  for (int64_t u = 0; u < d.nbu; ++u)
    if (up_col[u] != up_row[u]) low_cnt[up_col[u]]++;
  for (int64_t a = 0; a < na; ++a) row_ptr[a + 1] = row_ptr[a] + low_cnt[a] + (up_ptr[a + 1] - up_ptr[a]);
  d.nbf = row_ptr[na];
  std::vector<int32_t> col(d.nbf), up_full(d.nbu), up_mirror(d.nbu);
  {
    std::vector<int32_t> low_pos(na);
    for (int64_t a = 0; a < na; ++a) low_pos[a] = row_ptr[a];
    for (int64_t a = 0; a < na; ++a) {
      int32_t base = row_ptr[a] + low_cnt[a];
      for (int32_t u = up_ptr[a]; u < up_ptr[a + 1]; ++u) {
        int32_t b = up_col[u];
        int32_t pf = base + (u - up_ptr[a]);
        col[pf] = b;
        up_full[u] = pf;
        if (b == a) {
          up_mirror[u] = pf;
        } else {
          int32_t pm = low_pos[b]++;
          col[pm] = (int32_t)a;
          up_mirror[u] = pm;
        }
      }
    }
  }

  // ---- storage layout of S for the SpMV: every row's stored blocks padded to a multiple of 32 (the pads
  // have col = row and zero values), and inside each group of 32 blocks the 36 entries are interleaved
  // (entry e of the group's block l at e * 32 + l), so that a warp reads one entry of 32 blocks per
  // coalesced 128-byte load.  up_full / up_mirror hold positions in this padded order.
  std::vector<int32_t> prow_ptr(na + 1, 0), row_len(na);
  for (int64_t a = 0; a < na; ++a) {
    row_len[a] = row_ptr[a + 1] - row_ptr[a];
    prow_ptr[a + 1] = prow_ptr[a] + ((row_len[a] + 31) / 32) * 32;
  }
  d.nbp = prow_ptr[na];
  std::vector<int32_t> pcol(d.nbp);
  for (int64_t a = 0; a < na; ++a)
    for (int32_t k = 0; k < prow_ptr[a + 1] - prow_ptr[a]; ++k)
      pcol[prow_ptr[a] + k] = k < row_len[a] ? col[row_ptr[a] + k] : (int32_t)a;
  auto to_padded = [&](int32_t fp) {
    int64_t a = std::upper_bound(row_ptr.begin(), row_ptr.end(), fp) - row_ptr.begin() - 1;
    return prow_ptr[a] + (fp - row_ptr[a]);
  };
  for (int64_t u = 0; u < d.nbu; ++u) {
    up_full[u] = to_padded(up_full[u]);
    up_mirror[u] = to_padded(up_mirror[u]);
  }
  P.h_prow_ptr = prow_ptr;
  P.h_row_len = row_len;

  // ---- slot pairs per upper block (feature order inside a block), cut into work items
  std::vector<int64_t> pcount(d.nbu + 1, 0);
  auto find_up = [&](int32_t a, int32_t b) {
    auto it = std::lower_bound(up_col.begin() + up_ptr[a], up_col.begin() + up_ptr[a + 1], b);
    return (int32_t)(it - up_col.begin());
  };
  for (int64_t f = 0; f < d.nf; ++f)
    for (int32_t i = fslot_off[f]; i < fslot_off[f + 1]; ++i)
      for (int32_t j = i; j < fslot_off[f + 1]; ++j) pcount[find_up(slot_ent[i], slot_ent[j]) + 1]++;
  for (int64_t u = 0; u < d.nbu; ++u) pcount[u + 1] += pcount[u];
  d.npair = pcount[d.nbu];
  if (d.npair > (int64_t)INT32_MAX - 1) return fail(P, BA_ERR_ARG, "too many Schur pairs");
  std::vector<int32_t> pair_a(d.npair), pair_b(d.npair);
  {
    std::vector<int64_t> pos(pcount.begin(), pcount.end() - 1);
    for (int64_t f = 0; f < d.nf; ++f)
      for (int32_t i = fslot_off[f]; i < fslot_off[f + 1]; ++i)
        for (int32_t j = i; j < fslot_off[f + 1]; ++j) {
          int64_t q = pos[find_up(slot_ent[i], slot_ent[j])]++;
          pair_a[q] = i;
          // bit 31 marks a (camera slot, plane slot) pair of one feature: its direct block J_cam^T w J_plane
          const bool cam_plane = i != j && slot_type[i] == ENT_CAM && slot_type[j] == ENT_PLANE;
          pair_b[q] = (int32_t)((uint32_t)j | (cam_plane ? 0x80000000u : 0u));
        }
  }
  std::vector<int32_t> up_wi(d.nbu + 1, 0), wi_start;
  for (int64_t u = 0; u < d.nbu; ++u) {
    int64_t n = pcount[u + 1] - pcount[u];
    int64_t nw = (n + PAIR_CHUNK - 1) / PAIR_CHUNK;
    if (nw == 0) nw = 1;  // every block gets one (possibly empty) work item
    up_wi[u + 1] = up_wi[u] + (int32_t)nw;
    for (int64_t w = 0; w < nw; ++w) wi_start.push_back((int32_t)(pcount[u] + w * PAIR_CHUNK));
  }
  d.nwi = up_wi[d.nbu];
  wi_start.push_back((int32_t)d.npair);
  // a work item ends where the next starts, except at a block boundary
  std::vector<int32_t> wi_end(d.nwi);
  for (int64_t u = 0; u < d.nbu; ++u)
    for (int32_t w = up_wi[u]; w < up_wi[u + 1]; ++w)
      wi_end[w] = std::min<int64_t>(wi_start[w] + PAIR_CHUNK, pcount[u + 1]);
  // store start/end interleaved: wi_start[2w], wi_start[2w+1]
  std::vector<int32_t> wi_se(2 * d.nwi);
  for (int64_t w = 0; w < d.nwi; ++w) { wi_se[2 * w] = wi_start[w]; wi_se[2 * w + 1] = wi_end[w]; }

  // ---- permuted residual arrays
  std::vector<int8_t> rkind(nr);
  std::vector<int32_t> rcam(nr), rfeat(nr), rgrp(nr);
  std::vector<double> rmeas(4 * nr);
  for (int64_t j = 0; j < nr; ++j) {
    int32_t i = order[j];
    rkind[j] = kind[i]; rcam[j] = cam[i]; rfeat[j] = feat[i]; rgrp[j] = grp[i];
    for (int c = 0; c < 4; ++c) rmeas[4 * j + c] = meas[4 * i + c];
  }
  std::vector<uint8_t> ent_type(na);
  for (int64_t a = 0; a < na; ++a) ent_type[a] = a < d.nc ? ENT_CAM : (a < d.nc + d.npl ? ENT_PLANE : ENT_VP);

  // ---- upload
  ba_status s;
#define UP(dst, src) if ((s = upload(P, dst, src)) != BA_OK) return s
  UP(P.rkind, rkind); UP(P.rcam, rcam); UP(P.rfeat, rfeat); UP(P.rgrp, rgrp);
  UP(P.rslot_c, rslot_c); UP(P.rslot_g, rslot_g); UP(P.meas64, rmeas);
  UP(P.fres_off, fres_off); UP(P.fslot_off, fslot_off);
  UP(P.slot_ent, slot_ent); UP(P.slot_feat, slot_feat); UP(P.slot_type, slot_type);
  UP(P.feat_plane_slot, feat_plane_slot); UP(P.ent_type, ent_type);
  UP(P.row_ptr, prow_ptr); UP(P.col, pcol); UP(P.row_len, row_len);
  UP(P.up_row, up_row); UP(P.up_full, up_full); UP(P.up_mirror, up_mirror); UP(P.up_wi, up_wi);
  UP(P.pair_a, pair_a); UP(P.pair_b, pair_b); UP(P.wi_start, wi_se);
  UP(P.cam_fixed, P.h_fixed);
  for (int k = 0; k < 2; ++k) {
    auto& S_ = P.ps[k];
    UP(S_.cam, P.h_cam); UP(S_.pts, P.h_pts); UP(S_.lin, P.h_lin); UP(S_.pln, P.h_pln); UP(S_.vps, P.h_vps);
    S_.camD = P.dnew<double>(d.nc * CAM_STRIDE);
    S_.grpD = P.dnew<double>((d.npl + d.nv) * GRP_STRIDE);
    if (!S_.camD || !S_.grpD) return fail(P, BA_ERR_OOM, "device allocation failed");
  }
  P.cur = 0;
#undef UP
  CU(cudaStreamSynchronize(P.stream));
  return BA_OK;
}

}  // namespace ba
