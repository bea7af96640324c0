// C ABI of libba and the host orchestration of one LM step.
//
// Per step (all on the problem's stream, one host synchronisation per step plus
// one per batch of PCG iterations):
//   [relinearise only after an accepted step]  derive -> K1 linearize
//   K2 invert (lambda)  -> K3 Schur items / blocks -> K4 block-Jacobi
//   PCG init, then batches of {SpMV+dot, update+dots, p-update} until the device
//   stop flag is set -> K7 back-substitution + predicted decrease
//   K8 candidate x (+) delta, derive, FP64 cost -> K9 accept / reject, damping
// A rejected step keeps the linearisation and only re-damps (the Jacobians do not
// depend on lambda).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <array>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <type_traits>

#include "ba_internal.cuh"

using namespace ba;

static const int kMeasDim[N_KINDS] = {2, 4, 0, 4, 0, 4, 2, 0, 0, 0, 0, 0, 0, 0, 0, 4};

static ba_status set_err(ba_problem* p, ba_status s, const std::string& m) {
  if (p) p->err = m;
  return s;
}

#define CUDA_OR(p, x)                                                                    \
  do {                                                                                   \
    cudaError_t e_ = (x);                                                                \
    if (e_ != cudaSuccess) return set_err(p, BA_ERR_CUDA, std::string(#x ": ") + cudaGetErrorString(e_)); \
  } while (0)

void* ba_problem::dalloc(size_t bytes) {
  void* ptr = alloc.get(bytes);
  if (ptr) bufs.push_back({ptr, bytes});
  return ptr;
}

extern "C" void ba_default_options(ba_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = BA_FP64;
  o->w_point = 1.0; o->w_line = 1.0; o->w_group = 0.5; o->w_wire = 0.1; o->w_vp = 5e3;
  o->cauchy_px = 1.0; o->cauchy_vp = 0.2;
  o->lambda0 = 1e-4; o->lambda_min = 1e-12; o->lambda_max = 1e12;
  o->min_gain = 1e-3; o->rel_cost_tol = 1e-6; o->max_lm_iters = 20;
  o->pcg_rel_tol = 1e-6; o->pcg_max_iters = 1000;
  o->precond = BA_PRECOND_BLOCK_JACOBI;
  o->cuda_stream = nullptr;
  o->wait_budget_cycles = 2000000000LL;
  o->mixed_lambda_floor = 0.0;
  o->w_rel = 5e3;
  o->cauchy_rel = 0.2;
  o->cam_dof = 6;
  o->w_group3d = 1.0;
  o->cauchy_3d = 1.0;
  o->w_wire3d = 1.0;
}

extern "C" ba_status ba_create(const ba_options* opts, ba_problem** out) {
  if (!out) return BA_ERR_ARG;
  *out = nullptr;
  ba_problem* p = new (std::nothrow) ba_problem();
  if (!p) return BA_ERR_OOM;
  if (opts) p->opt = *opts; else ba_default_options(&p->opt);
  if (p->opt.precision != BA_FP64 && p->opt.precision != BA_MIXED) { delete p; return BA_ERR_ARG; }
  if (p->opt.precond != BA_PRECOND_BLOCK_JACOBI && p->opt.precond != BA_PRECOND_LEARNED) { delete p; return BA_ERR_ARG; }
  if (!(p->opt.pcg_rel_tol > 0) || p->opt.pcg_max_iters <= 0) { delete p; return BA_ERR_ARG; }
  if ((p->opt.dev_alloc == nullptr) != (p->opt.dev_free == nullptr)) { delete p; return BA_ERR_ARG; }
  if (p->opt.cam_dof != 6 && p->opt.cam_dof != 9) { delete p; return BA_ERR_ARG; }
  if (p->opt.precision == BA_MIXED) p->opt.lambda_min = std::max(p->opt.lambda_min, p->opt.mixed_lambda_floor);
  p->alloc.fa = p->opt.dev_alloc; p->alloc.ff = p->opt.dev_free; p->alloc.ctx = p->opt.alloc_ctx;
  p->stream = (cudaStream_t)p->opt.cuda_stream;
  if (cudaGetDevice(&p->device) != cudaSuccess) { cudaGetLastError(); delete p; return BA_ERR_CUDA; }
  static std::atomic<uint64_t> next_serial{1};
  p->serial = next_serial++;
  *out = p;
  return BA_OK;
}

static void release_batch_graph(ba_problem* p) {
  auto& g = p->bgraph;
  if (g.stream) cudaStreamSynchronize(g.stream);
  if (g.exec) cudaGraphExecDestroy(g.exec);
  if (g.graph) cudaGraphDestroy(g.graph);
  if (g.stream) cudaStreamDestroy(g.stream);
  p->alloc.put(g.desc);
  p->alloc.put(g.order);
  p->alloc.put(g.queue);
  g = ba_problem::BatchGraph();
}

extern "C" void ba_destroy(ba_problem* p) {
  if (!p) return;
  cudaStreamSynchronize(p->stream);
  release_batch_graph(p);
  p->release_obs();
  for (auto& b : p->bufs) p->alloc.put(b.p);
  p->bufs.clear();
  if (p->hS) cudaFreeHost(p->hS);
  for (auto& e : p->ev)
    if (e) cudaEventDestroy(e);
  if (p->side) { cudaStreamSynchronize(p->side); cudaStreamDestroy(p->side); }
  for (auto& e : p->sev)
    if (e) cudaEventDestroy(e);
  cudaGetLastError();
  delete p;
}

extern "C" const char* ba_last_error(const ba_problem* p) { return p ? p->err.c_str() : "null problem"; }

// ---------------------------------------------------------------------------
// adding data (host staging; device inputs are copied down first)
template <class X>
static ba_status fetch(ba_problem* p, int mem, const X* src, size_t n, std::vector<X>& dst) {
  size_t o = dst.size();
  dst.resize(o + n);
  if (n == 0) return BA_OK;
  if (!src) return set_err(p, BA_ERR_ARG, "null array");
  if (mem == BA_MEM_HOST) {
    std::memcpy(dst.data() + o, src, n * sizeof(X));
  } else if (mem == BA_MEM_DEVICE) {
    CUDA_OR(p, cudaMemcpyAsync(dst.data() + o, src, n * sizeof(X), cudaMemcpyDeviceToHost, p->stream));
    CUDA_OR(p, cudaStreamSynchronize(p->stream));
  } else {
    return set_err(p, BA_ERR_ARG, "mem must be BA_MEM_HOST or BA_MEM_DEVICE");
  }
  return BA_OK;
}

static ba_status check_add(ba_problem* p, int64_t n) {
  if (!p) return BA_ERR_ARG;
  if (p->frozen) return set_err(p, BA_ERR_STATE, "the structure is frozen after the first step");
  if (n < 0) return set_err(p, BA_ERR_ARG, "negative count");
  return BA_OK;
}

extern "C" ba_status ba_add_cameras(ba_problem* p, int64_t n, int mem, const double* quat_t, const double* fk,
                                    const double* pp, const uint8_t* fixed) {
  ba_status s = check_add(p, n);
  if (s) return s;
  std::vector<double> a, b, c;
  std::vector<uint8_t> fx;
  if ((s = fetch(p, mem, quat_t, 7 * n, a))) return s;
  if ((s = fetch(p, mem, fk, 3 * n, b))) return s;
  if ((s = fetch(p, mem, pp, 2 * n, c))) return s;
  if (fixed) { if ((s = fetch(p, mem, fixed, n, fx))) return s; } else fx.assign(n, 0);
  for (int64_t i = 0; i < n; ++i) {
    for (int k = 0; k < 7; ++k) p->h_cam.push_back(a[7 * i + k]);
    for (int k = 0; k < 3; ++k) p->h_cam.push_back(b[3 * i + k]);
    for (int k = 0; k < 2; ++k) p->h_cam.push_back(c[2 * i + k]);
    p->h_fixed.push_back((uint8_t)(fx[i] & 0x3F));
  }
  for (double v : p->h_cam)
    if (!std::isfinite(v)) return set_err(p, BA_ERR_ARG, "non-finite camera parameter");
  return BA_OK;
}

extern "C" ba_status ba_add_features(ba_problem* p, int kind, int64_t n, int mem, const double* params) {
  ba_status s = check_add(p, n);
  if (s) return s;
  if (kind == BA_POINT) s = fetch(p, mem, params, 3 * n, p->h_pts);
  else if (kind == BA_LINE) s = fetch(p, mem, params, 6 * n, p->h_lin);
  else return set_err(p, BA_ERR_ARG, "feature kind must be BA_POINT or BA_LINE");
  return s;
}

extern "C" ba_status ba_add_groups(ba_problem* p, int kind, int64_t n, int mem, const double* params) {
  ba_status s = check_add(p, n);
  if (s) return s;
  if (kind == BA_PLANE) s = fetch(p, mem, params, 4 * n, p->h_pln);
  else if (kind == BA_VP) s = fetch(p, mem, params, 3 * n, p->h_vps);
  else if (kind == BA_SPHERE) s = fetch(p, mem, params, 4 * n, p->h_sph);
  else if (kind == BA_CYLINDER) s = fetch(p, mem, params, 7 * n, p->h_cyl);
  else if (kind == BA_CONE) s = fetch(p, mem, params, 7 * n, p->h_cone);
  else if (kind == BA_ELLIPSOID) s = fetch(p, mem, params, 10 * n, p->h_ell);
  else if (kind == BA_CUBOID) s = fetch(p, mem, params, 10 * n, p->h_cub);
  else return set_err(p, BA_ERR_ARG, "unknown group kind");
  return s;
}

extern "C" ba_status ba_add_relations(ba_problem* p, int64_t n, int mem, const int32_t* kind_a, const int32_t* a,
                                      const int32_t* kind_b, const int32_t* b, const int32_t* type) {
  ba_status s = check_add(p, n);
  if (s) return s;
  if (n == 0) return BA_OK;
  if (!kind_a || !a || !kind_b || !b || !type) return set_err(p, BA_ERR_ARG, "null array");
  std::vector<int32_t> cols[5];
  const int32_t* src[5] = {kind_a, a, kind_b, b, type};
  for (int k = 0; k < 5; ++k)
    if ((s = fetch(p, mem, src[k], (size_t)n, cols[k]))) return s;
  const size_t o = p->h_rel.size();
  p->h_rel.resize(o + 5 * (size_t)n);
  for (int64_t i = 0; i < n; ++i)
    for (int k = 0; k < 5; ++k) p->h_rel[o + 5 * i + k] = cols[k][i];
  return BA_OK;
}

extern "C" ba_status ba_set_intrinsics(ba_problem* p, int64_t n_intr, int mem, const double* fk,
                                      const int32_t* intr_of_cam, int64_t n_cams) {
  ba_status s = check_add(p, n_intr);
  if (s) return s;
  if (p->opt.cam_dof != 9) return set_err(p, BA_ERR_ARG, "ba_set_intrinsics needs cam_dof = 9 (refined intrinsics)");
  if (n_cams < 0) return set_err(p, BA_ERR_ARG, "negative count");
  if ((n_intr && !fk) || (n_cams && !intr_of_cam)) return set_err(p, BA_ERR_ARG, "null array");
  std::vector<double> v;
  std::vector<int32_t> m;
  if ((s = fetch(p, mem, fk, 3 * (size_t)n_intr, v))) return s;
  if ((s = fetch(p, mem, intr_of_cam, (size_t)n_cams, m))) return s;
  for (double x : v)
    if (!std::isfinite(x)) return set_err(p, BA_ERR_ARG, "non-finite intrinsics value");
  for (int64_t i = 0; i < n_cams; ++i)
    if (m[i] < 0 || m[i] >= n_intr)
      return set_err(p, BA_ERR_ARG, "intr_of_cam[" + std::to_string(i) + "] out of range");
  p->h_intr = std::move(v);
  p->h_cam_k = std::move(m);
  p->intr_set = true;
  return BA_OK;
}

extern "C" ba_status ba_add_observations(ba_problem* p, int kind, int64_t n, int mem, const int32_t* cam,
                                         const int32_t* feature, const int32_t* other, const double* meas) {
  ba_status s = check_add(p, n);
  if (s) return s;
  if (kind < 0 || kind >= N_KINDS) return set_err(p, BA_ERR_ARG, "unknown observation kind");
  if (mem != BA_MEM_HOST && mem != BA_MEM_DEVICE) return set_err(p, BA_ERR_ARG, "mem must be BA_MEM_HOST or BA_MEM_DEVICE");
  if (n == 0) return BA_OK;
  const bool needs_other = kind == BA_OBS_PLANE_POINT || kind == BA_OBS_PLANE_LINE || kind == BA_OBS_VP ||
                           kind == BA_OBS_PLANE_POINT3D || kind == BA_OBS_PLANE_LINE3D || kind >= BA_OBS_SPHERE_POINT;
  const bool has_cam = res_has_cam(kind);
  const int md = kMeasDim[kind];
  if (!feature || (has_cam && !cam) || (md && !meas)) return set_err(p, BA_ERR_ARG, "null array");
  if (needs_other && !other) return set_err(p, BA_ERR_ARG, "this observation kind needs the group id array");
  // the records go straight to device memory: the structure build validates and merges them there
  ba_problem::ObsBatch b;
  b.kind = kind;
  b.md = md;
  b.n = n;
  const cudaMemcpyKind dir = mem == BA_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  bool ok = true;
  auto stage = [&](auto*& dst, const auto* src, size_t count) {
    if (!ok || !src) return;
    const size_t bytes = sizeof(*src) * count;
    dst = (std::remove_const_t<std::remove_reference_t<decltype(*src)>>*)p->alloc.get(bytes);
    if (!dst || cudaMemcpyAsync(dst, src, bytes, dir, p->stream) != cudaSuccess) ok = false;
  };
  stage(b.feat, feature, (size_t)n);
  if (has_cam) stage(b.cam, cam, (size_t)n);
  stage(b.other, other, (size_t)n);
  if (md) stage(b.meas, meas, (size_t)md * n);
  // the caller may reuse its buffers on return (also pinned ones, whose copies are asynchronous)
  const cudaError_t e = cudaStreamSynchronize(p->stream);
  if (!ok || e != cudaSuccess) {
    p->alloc.put(b.feat); p->alloc.put(b.cam); p->alloc.put(b.other); p->alloc.put(b.meas);
    cudaGetLastError();
    return set_err(p, ok ? BA_ERR_CUDA : BA_ERR_OOM, "could not copy the observations to the device");
  }
  p->d_obs.push_back(b);
  return BA_OK;
}

// ---------------------------------------------------------------------------
static bool mixed(const ba_problem* p) { return p->opt.precision == BA_MIXED; }

// Partition of the block rows of S over the CTAs of the persistent PCG kernel: rows are balanced by stored
// blocks (plus a small per-row term for the vector updates), and every row is cut into chunks of at most
// PCG_CHUNK blocks for the warps of its CTA.
static ba_status plan_pcg(ba_problem* p) {
  const Dims& d = p->d;
  std::vector<int32_t> rp(d.na + 1);
  CUDA_OR(p, cudaMemcpyAsync(rp.data(), p->row_ptr, sizeof(int32_t) * rp.size(), cudaMemcpyDeviceToHost, p->stream));
  CUDA_OR(p, cudaStreamSynchronize(p->stream));
  // rows are padded to multiples of 32 stored blocks: one chunk per 32 blocks (one block per lane)
  std::vector<int32_t> row_chunk0(d.na + 1, 0), chunk_beg;
  for (int64_t r = 0; r < d.na; ++r) {
    int32_t nch = (rp[r + 1] - rp[r]) / 32;
    for (int32_t k = 0; k < nch; ++k) chunk_beg.push_back(rp[r] + k * 32);
    row_chunk0[r + 1] = row_chunk0[r] + nch;
  }
  chunk_beg.push_back(rp[d.na]);
  int sms = 0, dev = 0;
  CUDA_OR(p, cudaGetDevice(&dev));
  CUDA_OR(p, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const bool mx = mixed(p);
  auto occ = [&](size_t smem) { return mx ? pcg_blocks_per_sm<float>(smem) : pcg_blocks_per_sm<double>(smem); };
  int per_sm = std::max(1, std::min(1, occ(48 * 1024)));
  // CTAs get contiguous runs of chunks of equal weight (32 blocks a chunk, 2 more for a chunk that opens
  // a row: the row's sums and vector updates); a long row may be cut between CTAs
  const int64_t Q = row_chunk0[d.na];
  std::vector<int32_t> cta_part;
  size_t smem = 0;
  for (int attempt = 0; attempt < 8; ++attempt) {
    const int64_t G = std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * per_sm, Q));
    const double total = 32.0 * (double)Q + 2.0 * (double)d.na;
    std::vector<int32_t> q0s(1, 0);
    double acc = 0;
    int64_t row = 0;
    for (int64_t q = 0; q < Q; ++q) {
      while (row_chunk0[row + 1] <= q) ++row;
      acc += 32.0 + (row_chunk0[row] == q ? 2.0 : 0.0);
      if ((int64_t)q0s.size() < G && acc >= total * (double)q0s.size() / (double)G && q + 1 < Q)
        q0s.push_back((int32_t)(q + 1));
    }
    while ((int64_t)q0s.size() < G + 1) q0s.push_back((int32_t)Q);
    cta_part.assign(4 * G, 0);
    int32_t maxrows = 1;
    int64_t rr = 0;
    for (int64_t c = 0; c < G; ++c) {
      const int32_t q0 = q0s[c], q1 = q0s[c + 1];
      int32_t t0 = 0, t1 = 0;
      if (q1 > q0) {
        while (row_chunk0[rr + 1] <= q0) ++rr;
        t0 = (int32_t)rr;
        int64_t re = rr;
        while (row_chunk0[re + 1] <= q1 - 1) ++re;
        t1 = (int32_t)(re + 1);
      }
      cta_part[4 * c] = q0; cta_part[4 * c + 1] = q1; cta_part[4 * c + 2] = t0; cta_part[4 * c + 3] = t1;
      maxrows = std::max(maxrows, t1 - t0);
    }
    // shared memory of the row sums: one segment of 6 double-width sums per (warp, row it touches)
    smem = sizeof(double) * 6 * ((size_t)maxrows + 16);
    if (smem > 72 * 1024) return set_err(p, BA_ERR_ARG, "reduced system too large or irregular for the PCG partition");
    if (mx) pcg_allow_smem<float>(smem); else pcg_allow_smem<double>(smem);
    if (occ(smem) >= per_sm) {
      p->pcg_grid = (int)G;
      break;
    }
    per_sm = std::max(1, per_sm - 1);
  }
  if (p->pcg_grid == 0) return set_err(p, BA_ERR_ARG, "no cooperative PCG launch configuration fits");
  p->pcg_smem = smem;
  ba_status s;
  auto up = [&](int32_t*& dst, const std::vector<int32_t>& v) -> ba_status {
    dst = p->dnew<int32_t>((int64_t)v.size());
    if (!dst) return set_err(p, BA_ERR_OOM, "device allocation failed");
    CUDA_OR(p, cudaMemcpyAsync(dst, v.data(), sizeof(int32_t) * v.size(), cudaMemcpyHostToDevice, p->stream));
    return BA_OK;
  };
  {
    // share of S kept in L2 across PCG iterations (fetched evict_last; the rest streams evict_first): about
    // half of the 126 MB L2, so that the vectors and the other kernels keep their share.  No persisting
    // set-aside is configured: reserving L2 for S slowed the linearisation and the whitening more than it
    // helped the PCG.
    constexpr double kKeepBytes = 60.0 * 1048576.0;
    const double sbytes = (double)Q * 32.0 * BS2 * (mx ? sizeof(float) : sizeof(double)) + (double)Q * 128.0;
    p->pcg_keep_frac = sbytes > 0 ? (float)std::min(1.0, kKeepBytes / sbytes) : 0.f;
  }
  p->pcg_carry = p->dnew<double>(6 * (int64_t)p->pcg_grid);
  if (!p->pcg_carry) return set_err(p, BA_ERR_OOM, "device allocation failed");
  if ((s = up(p->cta_part, cta_part))) return s;
  if ((s = up(p->row_chunk0, row_chunk0))) return s;
  if ((s = up(p->chunk_beg, chunk_beg))) return s;
  CUDA_OR(p, cudaStreamSynchronize(p->stream));
  return BA_OK;
}

// Partition of the typed storage's camera-row chunks over the CTAs of the persistent PCG (contiguous runs of
// equal arithmetic weight, a long camera row possibly cut between CTAs) and of the group rows (slices of
// equal size: their products are few, their sums of the CTAs' scatter are what they cost).
static ba_status plan_pcg_typed(ba_problem* p, const TypedPlan& tp) {
  const Dims& d = p->d;
  const int64_t nc = d.nc, ng = d.na - d.nc;
  int sms = 0, dev = 0;
  CUDA_OR(p, cudaGetDevice(&dev));
  CUDA_OR(p, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const bool mx = mixed(p);
  const int64_t Q = (int64_t)tp.chunks.size();
  const int64_t G = std::max<int64_t>(1, sms);
  std::vector<double> cw(Q + 1, 0.0);
  for (int64_t q = 0; q < Q; ++q) cw[q + 1] = cw[q] + tp.chunk_w[q];
  std::vector<int32_t> q0s(1, 0);
  for (int64_t q = 0; q < Q; ++q)
    if ((int64_t)q0s.size() < G && cw[q + 1] >= cw[Q] * (double)q0s.size() / (double)G && q + 1 < Q)
      q0s.push_back((int32_t)(q + 1));
  while ((int64_t)q0s.size() < G + 1) q0s.push_back((int32_t)Q);
  std::vector<int32_t> cta_part(4 * G, 0);
  int32_t maxrows = 1;
  int64_t rr = 0;
  for (int64_t c = 0; c < G; ++c) {
    const int32_t q0 = q0s[c], q1 = q0s[c + 1];
    int32_t t0 = 0, t1 = 0;
    if (q1 > q0) {
      while (tp.row_chunk0[rr + 1] <= q0) ++rr;
      t0 = (int32_t)rr;
      int64_t re = rr;
      while (tp.row_chunk0[re + 1] <= q1 - 1) ++re;
      t1 = (int32_t)(re + 1);
    }
    cta_part[4 * c] = q0; cta_part[4 * c + 1] = q1; cta_part[4 * c + 2] = t0; cta_part[4 * c + 3] = t1;
    maxrows = std::max(maxrows, t1 - t0);
  }
  // group rows in slices of about equal work: the row's group-group blocks plus its values' sums of the
  // CTAs' scatter
  std::vector<int32_t> gs(G + 1, (int32_t)ng);
  {
    std::vector<int32_t> ggp(ng + 1);
    if (ng) CUDA_OR(p, cudaMemcpy(ggp.data(), p->gg_ptr, sizeof(int32_t) * (ng + 1), cudaMemcpyDeviceToHost));
    else ggp[0] = 0;
    auto wrow = [&](int64_t g) { return (double)(ggp[g + 1] - ggp[g]) + 4.0; };
    double tot = 0;
    for (int64_t g = 0; g < ng; ++g) tot += wrow(g);
    gs[0] = 0;
    int64_t c = 1;
    double acc = 0;
    for (int64_t g = 0; g < ng && c < G; ++g) {
      acc += wrow(g);
      while (c < G && acc >= tot * (double)c / (double)G) gs[c++] = (int32_t)(g + 1);
    }
    for (; c <= G; ++c) gs[c] = (int32_t)ng;
    // the products of a slice's group-group blocks are staged in the group accumulators' shared memory
    int64_t maxgg = 0;
    for (int64_t c2 = 0; c2 < G; ++c2) maxgg = std::max<int64_t>(maxgg, ggp[gs[c2 + 1]] - ggp[gs[c2]]);
    const size_t gacc_bytes = mx ? pcg_typed_gacc_bytes<float>(p->gv) : pcg_typed_gacc_bytes<double>(p->gv);
    if ((size_t)maxgg * 6 * (mx ? 2 * sizeof(float) : sizeof(double)) > gacc_bytes)
      return set_err(p, BA_ERR_ARG, "group rows with too many group-group blocks for the typed PCG");
  }
  std::vector<int32_t> gvi(std::max(p->gv, 1), 0);
  for (int64_t g = 0; g < d.npl; ++g)
    for (int k = 0; k < 3; ++k) gvi[3 * g + k] = (int32_t)(6 * (nc + g) + k);
  for (int64_t v = 0; v < d.nv; ++v)
    for (int k = 0; k < 2; ++k) gvi[3 * d.npl + 2 * v + k] = (int32_t)(6 * (nc + d.npl + v) + k);
  for (int64_t q = 0; q < d.nk; ++q)
    for (int k = 0; k < 3; ++k) gvi[3 * d.npl + 2 * d.nv + 3 * q + k] = (int32_t)(6 * (nc + d.npl + d.nv + q) + k);
  // the owned values of every CTA (its whole camera rows and its group rows), kept in shared memory
  int64_t nown = 0;
  for (int64_t c = 0; c < G; ++c) {
    const int32_t q0 = cta_part[4 * c], t0 = cta_part[4 * c + 2], t1 = cta_part[4 * c + 3];
    const int32_t o0 = (t0 < t1 && tp.row_chunk0[t0] != q0) ? t0 + 1 : t0;
    nown = std::max<int64_t>(nown, 6 * ((int64_t)std::max(0, t1 - o0) + (gs[c + 1] - gs[c])));
  }
  nown = std::max<int64_t>(nown, 2);
  // shared memory: the fixed part (stage, group accumulators and operands), the owned vectors (6 doubles and 6
  // values of the block inverses per owned value) and one segment of 6 sums per (warp, camera row it touches)
  const size_t seg = (mx ? sizeof(float) * 2 : sizeof(double)) * 6 * ((size_t)maxrows + 16);
  const size_t own = sizeof(double) * 6 * (size_t)nown + (((mx ? sizeof(float) : sizeof(double)) * 6 * (size_t)nown + 15) & ~(size_t)15);
  const size_t smem = (mx ? pcg_typed_fixed_smem<float>(p->gv) : pcg_typed_fixed_smem<double>(p->gv)) + own + seg;
  p->pcg_nown = (int)nown;
  if (smem > 227 * 1024)
    return set_err(p, BA_ERR_ARG, "reduced system too large or irregular for the PCG partition");
  const int per_sm = mx ? pcg_typed_blocks_per_sm<float>(smem) : pcg_typed_blocks_per_sm<double>(smem);
  if (per_sm < 1) return set_err(p, BA_ERR_ARG, "no cooperative PCG launch configuration fits");
  p->pcg_grid = (int)G;
  p->pcg_smem = smem;
  {
    // share of S kept in L2 across PCG iterations (fetched evict_last; the rest streams evict_first)
    constexpr double kKeepBytes = 60.0 * 1048576.0;
    const double sbytes = (double)p->gg_val0 * (mx ? sizeof(float) : sizeof(double)) + 128.0 * (double)Q;
    p->pcg_keep_frac = sbytes > 0 ? (float)std::min(1.0, kKeepBytes / sbytes) : 0.f;
  }
  ba_status s;
  auto up = [&](int32_t*& dst, const std::vector<int32_t>& v) -> ba_status {
    dst = p->dnew<int32_t>((int64_t)v.size());
    if (!dst) return set_err(p, BA_ERR_OOM, "device allocation failed");
    CUDA_OR(p, cudaMemcpyAsync(dst, v.data(), sizeof(int32_t) * v.size(), cudaMemcpyHostToDevice, p->stream));
    return BA_OK;
  };
  p->pcg_carry = p->dnew<double>(6 * G);
  p->part_g = p->dnew<double>(G * std::max(p->gv, 1));
  p->tchunk = p->dnew<int4>(std::max<int64_t>(Q, 1));
  if (!p->pcg_carry || !p->part_g || !p->tchunk) return set_err(p, BA_ERR_OOM, "device allocation failed");
  if (Q) CUDA_OR(p, cudaMemcpyAsync(p->tchunk, tp.chunks.data(), sizeof(int4) * Q, cudaMemcpyHostToDevice, p->stream));
  if ((s = up(p->cta_part, cta_part))) return s;
  if ((s = up(p->row_chunk0, tp.row_chunk0))) return s;
  if ((s = up(p->cta_gs, gs))) return s;
  if ((s = up(p->gv_idx, gvi))) return s;
  CUDA_OR(p, cudaStreamSynchronize(p->stream));
  return BA_OK;
}

static ba_status freeze(ba_problem* p) {
  if (p->frozen) return BA_OK;
  if (p->h_cam.empty() && p->h_pts.empty() && p->h_lin.empty()) return set_err(p, BA_ERR_STATE, "empty problem");
  ba_status s = build_structure(*p);
  if (s) return s;
  p->frozen = true;
  const Dims& d = p->d;
  const size_t T = mixed(p) ? sizeof(float) : sizeof(double);
  p->gv = (int)(3 * d.npl + 2 * d.nv + 3 * d.nk);
  auto A = [&](void*& dst, size_t bytes) -> bool {
    dst = p->dalloc(bytes);
    return dst != nullptr;
  };
  bool ok = true;
  ok &= A(p->slotW, T * SW * (size_t)d.ne);
  ok &= A(p->slotZ, T * SW * (size_t)d.ne);
  ok &= A(p->slotG, T * SG * (size_t)d.ne);
  p->slotH = p->slotG ? (void*)((char*)p->slotG + T * HG_H) : nullptr;   // a view into the G|H records
  ok &= A(p->slotB, T * SB * (size_t)d.ne);
  ok &= A(p->slotC, T * SC * (size_t)d.ne);
  if (d.nk || d.nbx() || d.njp) ok &= A(p->slotCK, T * SC * (size_t)d.ne);
  if (d.ngs() || d.nbx()) ok &= A(p->slotCS, T * SCS * (size_t)d.ne);
  ok &= A(p->slotBS, T * SBS * (size_t)d.ne);
  ok &= A(p->Minv, T * BS2 * (size_t)d.na);
  p->featV = p->dnew<double>(10 * d.nf); p->featVinv = p->dnew<double>(10 * d.nf);
  p->featg = p->dnew<double>(4 * d.nf); p->featu = p->dnew<double>(4 * d.nf); p->dfeat = p->dnew<double>(4 * d.nf);
  p->featL = p->dnew<double>(10 * d.nf);
  ok &= p->featV && p->featVinv && p->featg && p->featu && p->dfeat && p->featL;
  double** vecs[] = {&p->bvec, &p->Dg, &p->x, &p->r, &p->z, &p->p, &p->Ap, &p->sdiag, &p->svec};
  for (double** v : vecs) { *v = p->dnew<double>(6 * d.na); ok &= *v != nullptr; }
  int64_t maxb = std::max<int64_t>({(d.nr + 255) / 256, (d.nfp + 127) / 128, (d.na * 32 + 255) / 256, (d.na + 127) / 128,
                                    4 * 148 * 4, 1});
  p->red = p->dnew<double>(2 * maxb + 16);
  p->S = p->dnew<DevScalars>(1);
  ok &= p->red && p->S;
  if (mixed(p)) {
    ok &= A(*(void**)&p->phl, sizeof(float2) * 6 * (size_t)d.na);
    ok &= A(p->camT, sizeof(float) * CAM_STRIDE * (size_t)d.nc);
    ok &= A(p->grpT, sizeof(float) * GRP_STRIDE * (size_t)(d.npl + d.nv));
    ok &= A(p->ptsT, sizeof(float) * 3 * (size_t)d.np);
    ok &= A(p->linT, sizeof(float) * 6 * (size_t)d.nl);
    ok &= A(p->measT, sizeof(float) * 4 * (size_t)d.nr);
    if (d.ngs()) ok &= A(p->srfT, sizeof(float) * SRF_STRIDE * (size_t)d.ngs());
    if (d.nbx()) ok &= A(p->bxT, sizeof(float) * BOX_STRIDE * (size_t)d.nbx());
  }
  if (!ok) return set_err(p, BA_ERR_OOM, "device allocation failed");
  // one-time zero fill of the slot and feature arrays
  CUDA_OR(p, cudaMemsetAsync(p->slotW, 0, T * SW * (size_t)d.ne, p->stream));
  CUDA_OR(p, cudaMemsetAsync(p->slotC, 0, T * SC * (size_t)d.ne, p->stream));
  if (d.nk || d.nbx() || d.njp) CUDA_OR(p, cudaMemsetAsync(p->slotCK, 0, T * SC * (size_t)d.ne, p->stream));
  if (d.ngs() || d.nbx()) CUDA_OR(p, cudaMemsetAsync(p->slotCS, 0, T * SCS * (size_t)d.ne, p->stream));
  CUDA_OR(p, cudaMemsetAsync(p->dfeat, 0, sizeof(double) * 4 * (size_t)d.nf, p->stream));
  CUDA_OR(p, cudaMemsetAsync(p->x, 0, sizeof(double) * 6 * (size_t)d.na, p->stream));
  // float copy of the measurements for the mixed-precision linearisation, on the device
  if (mixed(p) && d.nr) CUDA_OR(p, launch_convert(p->stream, 4 * d.nr, p->meas64, (float*)p->measT));
  CUDA_OR(p, cudaMallocHost((void**)&p->hS, sizeof(DevScalars)));
  std::memset(p->hS, 0, sizeof(DevScalars));
  p->hS->lambda = p->opt.lambda0;
  p->hS->nu = 2.0;
  p->hS->max_iters = p->opt.pcg_max_iters;
  CUDA_OR(p, cudaMemcpyAsync(p->S, p->hS, sizeof(DevScalars), cudaMemcpyHostToDevice, p->stream));
  for (auto& e : p->ev) CUDA_OR(p, cudaEventCreate(&e));
  // the second stream of the candidate's linearisation (beside the FP64 cost pass)
  CUDA_OR(p, cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking));
  for (auto& e : p->sev) CUDA_OR(p, cudaEventCreate(&e));
  // cost at the initial parameters
  CUDA_OR(p, ensure_ln1p_table(p->stream));
  if (mixed(p)) launch_prepare<float>(*p, false); else launch_prepare<double>(*p, false);
  launch_cost(*p, false);
  launch_rel_cost(*p, false);
  CUDA_OR(p, cudaGetLastError());
  CUDA_OR(p, cudaMemcpyAsync(p->hS, p->S, sizeof(DevScalars), cudaMemcpyDeviceToHost, p->stream));
  CUDA_OR(p, cudaStreamSynchronize(p->stream));
  return BA_OK;
}

// The storage of S and the PCG partition, made when S is first built.  A window of ba_solve_batch
// (for_batch), whose single-CTA kernels read S in full (both triangles, 6 x 6), keeps the full storage; a
// problem stepped on its own takes the typed storage when its group values fit (see TY_CC).
static ba_status ensure_sstore(ba_problem* p, bool for_batch) {
  if (p->Sval) return BA_OK;
  const Dims& d = p->d;
  const size_t T = mixed(p) ? sizeof(float) : sizeof(double);
  // spheres, cylinders and cones keep the full storage (their camera blocks are 4 to 6 wide)
  p->typed = !for_batch && d.nc > 0 && d.ngs() == 0 && d.nbx() == 0 && d.njp == 0 &&
             3 * d.npl + 2 * d.nv + 3 * d.nk <= GV_MAX;
  ba_status s;
  if (p->typed) {
    TypedPlan tplan;
    if ((s = build_typed_storage(*p, tplan))) return s;
    // a partition whose shared memory does not fit (very many short camera rows on one CTA) takes the full
    // storage instead
    if (plan_pcg_typed(p, tplan) != BA_OK) {
      if (p->pcg_grid) return BA_ERR_OOM;
      p->typed = false;
      p->err.clear();
    }
  }
  if (!p->typed && (s = plan_pcg(p))) return s;
  const size_t nsval = p->typed ? (size_t)p->tvals : (size_t)BS2 * d.nbp;
  p->Sval = p->dalloc(T * nsval);
  if (!p->Sval) return set_err(p, BA_ERR_OOM, "device allocation failed");
  CUDA_OR(p, cudaMemsetAsync(p->Sval, 0, T * nsval, p->stream));
  return BA_OK;
}

static ba_status sync_scalars(ba_problem* p) {
  CUDA_OR(p, cudaGetLastError());
  CUDA_OR(p, cudaMemcpyAsync(p->hS, p->S, sizeof(DevScalars), cudaMemcpyDeviceToHost, p->stream));
  CUDA_OR(p, cudaStreamSynchronize(p->stream));
  if (p->hS->flags & PCG_FLAG_TIMEOUT) {
    // a bounded wait of the PCG kernel ran out: a grid barrier (wait_budget_cycles) or a bulk copy of S
    const int cleared = p->hS->flags & ~PCG_FLAG_TIMEOUT;
    CUDA_OR(p, cudaMemcpy(&p->S->flags, &cleared, sizeof(int), cudaMemcpyHostToDevice));
    return set_err(p, BA_ERR_TIMEOUT, "PCG: a bounded device wait (grid barrier or copy of S) ran out");
  }
  return BA_OK;
}

// events: ev[0] start, ev[1+k] end of kernel stage k (k = 0..9, see ba_step_report.ms_kernel)
#define MARK(k) CUDA_OR(p, cudaEventRecord(p->ev[1 + (k)], p->stream))

template <class T>
static ba_status build_reduced_t(ba_problem* p, double lambda, bool* relin) {
  ba_status s0 = ensure_sstore(p, false);
  if (s0) return s0;
  if (!p->have_lin) {
    launch_prepare<T>(*p, false);
    launch_linearize<T>(*p);
    launch_rel_linearize(*p);
    p->have_lin = true;
    p->spec_lin = false;
    if (relin) *relin = true;
  }
  MARK(0);
  launch_invert<T>(*p, lambda);
  MARK(1);
  launch_schur<T>(*p, lambda);  // records ev[3] between the item and the block pass
  launch_rel_offdiag<T>(*p);
  MARK(3);
  CUDA_OR(p, cudaGetLastError());
  p->have_reduced = true;
  p->last_lambda = lambda;
  return BA_OK;
}

template <class T>
static void build_precond_t(ba_problem* p) {
  if (p->opt.precond == BA_PRECOND_LEARNED && p->pre_ready) launch_pre_learned<T>(*p);
  else launch_precond<T>(*p);
}

template <class T>
static ba_status solve_reduced_t(ba_problem* p) {
  build_precond_t<T>(p);
  MARK(4);
  launch_pcg<T>(*p);
  if (p->pcg_err != cudaSuccess) return set_err(p, BA_ERR_CUDA, std::string("PCG launch: ") + cudaGetErrorString(p->pcg_err));
  MARK(5);
  launch_backsub<T>(*p);
  launch_rel_pred(*p);
  MARK(6);
  CUDA_OR(p, cudaGetLastError());
  return BA_OK;
}

template <class T>
static ba_status lm_step_t(ba_problem* p, ba_step_report* rep) {
  const double lam = p->hS->lambda;
  bool relin = false;
  const bool relin_spec = p->have_lin && p->spec_lin;   // this step's Jacobians were made by the previous step
  p->launches = 0;
  CUDA_OR(p, cudaEventRecord(p->ev[0], p->stream));
  ba_status s = build_reduced_t<T>(p, lam, &relin);
  if (s) return s;
  if ((s = solve_reduced_t<T>(p))) return s;
  launch_candidate(*p);
  launch_prepare<T>(*p, true);
  MARK(7);
  // The next step linearises at the candidate whenever this one accepts it (most steps): do it now, on the
  // second stream, while the FP64 cost pass (FP64 pipe) evaluates the candidate; a rejection discards it.
  const bool spec = p->side != nullptr;
  if (spec) {
    CUDA_OR(p, cudaEventRecord(p->sev[0], p->stream));
    CUDA_OR(p, cudaStreamWaitEvent(p->side, p->sev[0], 0));
    cudaStream_t main_stream = p->stream;
    p->stream = p->side;
    p->cur ^= 1;   // the candidate's parameter set
    cudaEventRecord(p->sev[1], p->stream);
    launch_prepare<T>(*p, false, true);
    launch_linearize<T>(*p);
    launch_rel_linearize(*p);
    cudaEventRecord(p->sev[2], p->stream);
    p->cur ^= 1;
    p->stream = main_stream;
  }
  launch_cost(*p, true);
  launch_rel_cost(*p, true);
  MARK(8);
  launch_decide(*p);
  MARK(9);
  if (spec) CUDA_OR(p, cudaStreamWaitEvent(p->stream, p->sev[2], 0));
  if ((s = sync_scalars(p))) return s;
  DevScalars& h = *p->hS;
  ba_step_report r;
  std::memset(&r, 0, sizeof(r));
  r.cost = h.E; r.cost_px = h.Epx; r.cost_new = h.Enew; r.cost_px_new = h.Epxnew;
  r.pred = h.pred; r.gain = h.gain; r.lambda = lam;
  r.pcg_iters = h.iters; r.pcg_rel = h.bnorm2 > 0 ? std::sqrt(h.rr / h.bnorm2) : 0.0;
  r.accepted = h.accepted; r.relinearized = (relin || relin_spec) ? 1 : 0;
  r.n_launches = p->launches;
  r.precond_fallbacks = -1;
  if (p->opt.precond == BA_PRECOND_LEARNED && p->pre_ready)
    CUDA_OR(p, cudaMemcpy(&r.precond_fallbacks, p->pre_fallbacks, sizeof(int), cudaMemcpyDeviceToHost));
  for (int k = 0; k < 10; ++k) cudaEventElapsedTime(&r.ms_kernel[k], p->ev[k], p->ev[k + 1]);
  if (p->spec_lin && relin_spec) r.ms_kernel[0] = p->spec_ms;   // made during the previous step
  float spec_ms = 0.f;
  if (spec) cudaEventElapsedTime(&spec_ms, p->sev[1], p->sev[2]);
  r.ms_linearize = r.ms_kernel[0];
  r.ms_schur = r.ms_kernel[1] + r.ms_kernel[2] + r.ms_kernel[3] + r.ms_kernel[4];
  r.ms_pcg = r.ms_kernel[5];
  r.ms_update = r.ms_kernel[6] + r.ms_kernel[7] + r.ms_kernel[8] + r.ms_kernel[9];
  p->spec_lin = spec;
  p->spec_ms = spec_ms;
  if (h.accepted) {
    double rel = std::fabs(h.Epx - h.Epxnew) / std::max(h.Epx, 1e-300);
    r.converged = rel < p->opt.rel_cost_tol ? 1 : 0;
    p->cur ^= 1;
    p->have_lin = spec;   // the candidate's linearisation is the new point's
    p->have_reduced = false;
    // the accepted cost becomes the current cost
    h.E = h.Enew; h.Epx = h.Epxnew;
    CUDA_OR(p, cudaMemcpyAsync(&p->S->E, &h.E, 2 * sizeof(double), cudaMemcpyHostToDevice, p->stream));
  } else {
    // the slot records now hold the candidate's linearisation: the next step linearises the current point again
    if (spec) p->have_lin = false;
    if (lam >= p->opt.lambda_max) {
      // rejected at the largest damping: no step lowers the cost at the working precision (the analogue of
      // a trust region shrunk to its minimum radius), so the iteration has converged
      r.converged = 1;
    }
  }
  if (rep) *rep = r;
  if (!std::isfinite(h.E)) return set_err(p, BA_ERR_NUMERIC, "non-finite cost");
  return BA_OK;
}

extern "C" ba_status ba_lm_step(ba_problem* p, ba_step_report* out) {
  if (!p) return BA_ERR_ARG;
  ba_status s = freeze(p);
  if (s) return s;
  return mixed(p) ? lm_step_t<float>(p, out) : lm_step_t<double>(p, out);
}

extern "C" ba_status ba_solve(ba_problem* p, ba_solve_report* out) {
  if (!p) return BA_ERR_ARG;
  auto t0 = std::chrono::steady_clock::now();
  ba_status s = freeze(p);
  if (s) return s;
  auto t1 = std::chrono::steady_clock::now();
  ba_solve_report r;
  std::memset(&r, 0, sizeof(r));
  r.cost0 = p->hS->E;
  for (int it = 0; it < p->opt.max_lm_iters; ++it) {
    ba_step_report sr;
    if ((s = ba_lm_step(p, &sr))) return s;
    r.iters++;
    r.total_pcg_iters += sr.pcg_iters;
    if (sr.accepted) r.accepted_steps++;
    if (sr.converged) { r.converged = 1; break; }
  }
  r.cost = p->hS->E;
  r.cost_px = p->hS->Epx;
  auto t2 = std::chrono::steady_clock::now();
  r.ms_structure = std::chrono::duration<double, std::milli>(t1 - t0).count();
  r.ms_total = std::chrono::duration<double, std::milli>(t2 - t0).count();
  if (out) *out = r;
  return BA_OK;
}

// ---------------------------------------------------------------------------
template <class X>
static ba_status put_out(ba_problem* p, int mem, X* dst, const X* src, size_t n) {
  if (n == 0) return BA_OK;
  if (!dst) return set_err(p, BA_ERR_ARG, "null output");
  cudaMemcpyKind k = mem == BA_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  CUDA_OR(p, cudaMemcpyAsync(dst, src, n * sizeof(X), k, p->stream));
  CUDA_OR(p, cudaStreamSynchronize(p->stream));
  return BA_OK;
}

extern "C" ba_status ba_get_cameras(ba_problem* p, int mem, double* quat_t) {
  if (!p) return BA_ERR_ARG;
  ba_status s = freeze(p);
  if (s) return s;
  const int64_t n = p->d.nc;
  std::vector<double> h(12 * n);
  if ((s = put_out(p, BA_MEM_HOST, h.data(), p->ps[p->cur].cam, h.size()))) return s;
  std::vector<double> o(7 * n);
  for (int64_t i = 0; i < n; ++i)
    for (int k = 0; k < 7; ++k) o[7 * i + k] = h[12 * i + k];
  if (mem == BA_MEM_HOST) { if (n) std::memcpy(quat_t, o.data(), o.size() * sizeof(double)); return BA_OK; }
  CUDA_OR(p, cudaMemcpy(quat_t, o.data(), o.size() * sizeof(double), cudaMemcpyHostToDevice));
  return BA_OK;
}

extern "C" ba_status ba_get_features(ba_problem* p, int kind, int mem, double* params) {
  if (!p) return BA_ERR_ARG;
  ba_status s = freeze(p);
  if (s) return s;
  if (kind == BA_POINT) return put_out(p, mem, params, (const double*)p->ps[p->cur].pts, 3 * (size_t)p->d.np);
  if (kind == BA_LINE) return put_out(p, mem, params, (const double*)p->ps[p->cur].lin, 6 * (size_t)p->d.nl);
  return set_err(p, BA_ERR_ARG, "bad feature kind");
}

extern "C" ba_status ba_get_groups(ba_problem* p, int kind, int mem, double* params) {
  if (!p) return BA_ERR_ARG;
  ba_status s = freeze(p);
  if (s) return s;
  if (kind == BA_PLANE) return put_out(p, mem, params, (const double*)p->ps[p->cur].pln, 4 * (size_t)p->d.npl);
  if (kind == BA_VP) return put_out(p, mem, params, (const double*)p->ps[p->cur].vps, 3 * (size_t)p->d.nv);
  if (kind == BA_SPHERE || kind == BA_CYLINDER || kind == BA_CONE) {
    // the surface records (SRF_STRIDE values) in the add layout: sphere 4, cylinder 7, cone 7 values
    const Dims& d = p->d;
    const int64_t g0 = kind == BA_SPHERE ? 0 : kind == BA_CYLINDER ? d.nsp : d.nsp + d.ncy;
    const int64_t n = kind == BA_SPHERE ? d.nsp : kind == BA_CYLINDER ? d.ncy : d.nco;
    const int w = kind == BA_SPHERE ? 4 : 7;
    if (n == 0) return BA_OK;
    std::vector<double> h(SRF_STRIDE * n), o(w * n);
    ba_status st = put_out(p, BA_MEM_HOST, h.data(), (const double*)p->ps[p->cur].srf + SRF_STRIDE * g0, h.size());
    if (st) return st;
    for (int64_t i = 0; i < n; ++i)
      for (int k = 0; k < w; ++k) o[w * i + k] = h[SRF_STRIDE * i + k];
    if (!params) return set_err(p, BA_ERR_ARG, "null output");
    if (mem == BA_MEM_HOST) { std::memcpy(params, o.data(), o.size() * sizeof(double)); return BA_OK; }
    CUDA_OR(p, cudaMemcpy(params, o.data(), o.size() * sizeof(double), cudaMemcpyHostToDevice));
    return BA_OK;
  }
  if (kind == BA_ELLIPSOID || kind == BA_CUBOID) {
    // the 9-parameter records (R row-major, then 6 values) in the add layout: unit quaternion (w >= 0), 6 values
    const Dims& d = p->d;
    const int64_t g0 = kind == BA_ELLIPSOID ? 0 : d.nel, n = kind == BA_ELLIPSOID ? d.nel : d.ncu;
    if (n == 0) return BA_OK;
    std::vector<double> h(BOX_STRIDE * n), o(10 * n);
    ba_status st = put_out(p, BA_MEM_HOST, h.data(), (const double*)p->ps[p->cur].bx + BOX_STRIDE * g0, h.size());
    if (st) return st;
    for (int64_t i = 0; i < n; ++i) {
      const double* R = &h[BOX_STRIDE * i];
      double q[4];
      const double tr = R[0] + R[4] + R[8];
      if (tr > 0) {
        const double s4 = std::sqrt(tr + 1.0) * 2;
        q[0] = 0.25 * s4; q[1] = (R[7] - R[5]) / s4; q[2] = (R[2] - R[6]) / s4; q[3] = (R[3] - R[1]) / s4;
      } else if (R[0] > R[4] && R[0] > R[8]) {
        const double s4 = std::sqrt(1.0 + R[0] - R[4] - R[8]) * 2;
        q[0] = (R[7] - R[5]) / s4; q[1] = 0.25 * s4; q[2] = (R[1] + R[3]) / s4; q[3] = (R[2] + R[6]) / s4;
      } else if (R[4] > R[8]) {
        const double s4 = std::sqrt(1.0 + R[4] - R[0] - R[8]) * 2;
        q[0] = (R[2] - R[6]) / s4; q[1] = (R[1] + R[3]) / s4; q[2] = 0.25 * s4; q[3] = (R[5] + R[7]) / s4;
      } else {
        const double s4 = std::sqrt(1.0 + R[8] - R[0] - R[4]) * 2;
        q[0] = (R[3] - R[1]) / s4; q[1] = (R[2] + R[6]) / s4; q[2] = (R[5] + R[7]) / s4; q[3] = 0.25 * s4;
      }
      const double sg = q[0] < 0 ? -1.0 : 1.0;
      for (int k = 0; k < 4; ++k) o[10 * i + k] = sg * q[k];
      for (int k = 0; k < 6; ++k) o[10 * i + 4 + k] = h[BOX_STRIDE * i + 9 + k];
    }
    if (!params) return set_err(p, BA_ERR_ARG, "null output");
    if (mem == BA_MEM_HOST) { std::memcpy(params, o.data(), o.size() * sizeof(double)); return BA_OK; }
    CUDA_OR(p, cudaMemcpy(params, o.data(), o.size() * sizeof(double), cudaMemcpyHostToDevice));
    return BA_OK;
  }
  return set_err(p, BA_ERR_ARG, "bad group kind");
}

extern "C" ba_status ba_get_intrinsics(ba_problem* p, int mem, double* fk) {
  if (!p) return BA_ERR_ARG;
  ba_status s = freeze(p);
  if (s) return s;
  const int64_t n = p->d.nc;
  std::vector<double> h(12 * n);
  if ((s = put_out(p, BA_MEM_HOST, h.data(), p->ps[p->cur].cam, h.size()))) return s;
  std::vector<double> o(3 * n);
  for (int64_t i = 0; i < n; ++i)
    for (int k = 0; k < 3; ++k) o[3 * i + k] = h[12 * i + 7 + k];
  if (n == 0) return BA_OK;
  if (!fk) return set_err(p, BA_ERR_ARG, "null output");
  if (mem == BA_MEM_HOST) { std::memcpy(fk, o.data(), o.size() * sizeof(double)); return BA_OK; }
  CUDA_OR(p, cudaMemcpy(fk, o.data(), o.size() * sizeof(double), cudaMemcpyHostToDevice));
  return BA_OK;
}

extern "C" ba_status ba_intrinsics_count(ba_problem* p, int64_t* n) {
  if (!p || !n) return BA_ERR_ARG;
  ba_status s = freeze(p);
  if (s) return s;
  *n = p->d.nk;
  return BA_OK;
}

extern "C" ba_status ba_get_step_intrinsics(ba_problem* p, double* dk) {
  if (!p) return BA_ERR_ARG;
  if (!p->frozen) return set_err(p, BA_ERR_STATE, "no step computed");
  const Dims& d = p->d;
  if (d.nk == 0) return BA_OK;
  if (!dk) return set_err(p, BA_ERR_ARG, "null output");
  std::vector<double> x(6 * (size_t)d.nk);
  ba_status s;
  if ((s = put_out(p, BA_MEM_HOST, x.data(), (const double*)p->x + 6 * d.kbase(), x.size()))) return s;
  for (int64_t k = 0; k < d.nk; ++k)
    for (int j = 0; j < 3; ++j) dk[3 * k + j] = x[6 * k + j];
  return BA_OK;
}

extern "C" ba_status ba_get_lm_state(ba_problem* p, double* ln) {
  if (!p || !ln) return BA_ERR_ARG;
  if (!p->frozen) { ln[0] = p->opt.lambda0; ln[1] = 2.0; return BA_OK; }
  ln[0] = p->hS->lambda; ln[1] = p->hS->nu;
  return BA_OK;
}

extern "C" ba_status ba_set_lm_state(ba_problem* p, const double* ln) {
  if (!p || !ln || !(ln[0] > 0) || !(ln[1] > 0)) return p ? set_err(p, BA_ERR_ARG, "lambda and nu must be positive") : BA_ERR_ARG;
  ba_status s = freeze(p);
  if (s) return s;
  p->hS->lambda = ln[0]; p->hS->nu = ln[1];
  CUDA_OR(p, cudaMemcpyAsync(&p->S->lambda, &p->hS->lambda, 2 * sizeof(double), cudaMemcpyHostToDevice, p->stream));
  CUDA_OR(p, cudaStreamSynchronize(p->stream));
  return BA_OK;
}

extern "C" ba_status ba_eval_cost(ba_problem* p, double* cost, double* cost_px) {
  if (!p) return BA_ERR_ARG;
  ba_status s = freeze(p);
  if (s) return s;
  if (cost) *cost = p->hS->E;
  if (cost_px) *cost_px = p->hS->Epx;
  return BA_OK;
}

extern "C" ba_status ba_eval_log1p(int64_t n, const double* x, double* y, void* cuda_stream) {
  if (n < 0 || (n > 0 && (!x || !y))) return BA_ERR_ARG;
  if (n == 0) return BA_OK;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (launch_ln1p_eval(st, n, x, y) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return BA_ERR_CUDA;
  }
  return BA_OK;
}

extern "C" ba_status ba_measure_fma_rate(int precision, double* tflops, void* cuda_stream) {
  if (!tflops || (precision != BA_FP64 && precision != BA_MIXED)) return BA_ERR_ARG;
  if (fma_probe(precision, tflops, (cudaStream_t)cuda_stream) != cudaSuccess) {
    cudaGetLastError();
    return BA_ERR_CUDA;
  }
  return BA_OK;
}

extern "C" ba_status ba_build_reduced(ba_problem* p, double lambda) {
  if (!p) return BA_ERR_ARG;
  if (!(lambda >= 0) || !std::isfinite(lambda)) return set_err(p, BA_ERR_ARG, "lambda must be finite and >= 0");
  ba_status s = freeze(p);
  if (s) return s;
  s = mixed(p) ? build_reduced_t<float>(p, lambda, nullptr) : build_reduced_t<double>(p, lambda, nullptr);
  if (s) return s;
  CUDA_OR(p, cudaStreamSynchronize(p->stream));
  return BA_OK;
}

extern "C" ba_status ba_reduced_size(ba_problem* p, int64_t* nrows, int64_t* nnzb) {
  if (!p) return BA_ERR_ARG;
  ba_status s = freeze(p);
  if (s) return s;
  if (nrows) *nrows = p->d.na;
  if (nnzb) *nnzb = p->d.nbf;
  return BA_OK;
}

extern "C" ba_status ba_export_reduced_system(ba_problem* p, int32_t* row_ptr, int32_t* cols, double* vals, double* b) {
  if (!p) return BA_ERR_ARG;
  if (!p->have_reduced) return set_err(p, BA_ERR_STATE, "no reduced system built (call ba_build_reduced)");
  const Dims& d = p->d;
  ba_status s;
  // the device storage is padded (full or typed, see SView); the export is plain block-CSR of every block,
  // both triangles, 6 x 6
  std::vector<int32_t> pc(d.nbp), hsel;
  if ((s = put_out(p, BA_MEM_HOST, pc.data(), (const int32_t*)p->col, d.nbp))) return s;
  std::vector<double> pv;
  const size_t nsval = p->typed ? (size_t)p->tvals : (size_t)BS2 * d.nbp;
  if (vals) {
    pv.resize(nsval);
    if (mixed(p)) {
      std::vector<float> h(pv.size());
      if ((s = put_out(p, BA_MEM_HOST, h.data(), (const float*)p->Sval, h.size()))) return s;
      for (size_t i = 0; i < h.size(); ++i) pv[i] = h[i];
    } else if ((s = put_out(p, BA_MEM_HOST, pv.data(), (const double*)p->Sval, pv.size()))) {
      return s;
    }
    if (p->typed) {
      hsel.resize(d.nbp);
      if ((s = put_out(p, BA_MEM_HOST, hsel.data(), (const int32_t*)p->sel, d.nbp))) return s;
    }
  }
  SView hv;
  if (p->typed) {
    hv.sel = hsel.data(); hv.col = pc.data(); hv.nc = d.nc; hv.npl = d.npl; hv.gg_val0 = p->gg_val0;
    hv.kb = d.kbase();
  }
  int64_t o = 0;
  if (row_ptr) row_ptr[0] = 0;
  for (int64_t a = 0; a < d.na; ++a) {
    for (int32_t k = 0; k < p->h_row_len[a]; ++k, ++o) {
      const int64_t q = p->h_prow_ptr[a] + k;
      if (cols) cols[o] = pc[q];
      if (vals) {
        double blk[36];
        sview_load(hv, pv.data(), q, a, blk);
        for (int e = 0; e < BS2; ++e) vals[(size_t)o * BS2 + e] = blk[e];
      }
    }
    if (row_ptr) row_ptr[a + 1] = (int32_t)o;
  }
  if (b && (s = put_out(p, BA_MEM_HOST, b, (const double*)p->bvec, 6 * (size_t)d.na))) return s;
  return BA_OK;
}

extern "C" ba_status ba_compute_step(ba_problem* p, double* dcam, double* dplane, double* dvp, double* dpoint,
                                     double* dline, int* pcg_iters, double* pcg_rel, double* pred) {
  if (!p) return BA_ERR_ARG;
  if (!p->have_reduced) return set_err(p, BA_ERR_STATE, "no reduced system built (call ba_build_reduced)");
  ba_status s = mixed(p) ? solve_reduced_t<float>(p) : solve_reduced_t<double>(p);
  if (s) return s;
  if ((s = sync_scalars(p))) return s;
  const Dims& d = p->d;
  std::vector<double> x(6 * d.na), df(4 * d.nf);
  if ((s = put_out(p, BA_MEM_HOST, x.data(), (const double*)p->x, x.size()))) return s;
  if ((s = put_out(p, BA_MEM_HOST, df.data(), (const double*)p->dfeat, df.size()))) return s;
  if (dcam) for (int64_t i = 0; i < d.nc; ++i) for (int k = 0; k < 6; ++k) dcam[6 * i + k] = x[6 * i + k];
  if (dplane) for (int64_t i = 0; i < d.npl; ++i) for (int k = 0; k < 3; ++k) dplane[3 * i + k] = x[6 * (d.nc + i) + k];
  if (dvp) for (int64_t i = 0; i < d.nv; ++i) for (int k = 0; k < 2; ++k) dvp[2 * i + k] = x[6 * (d.nc + d.npl + i) + k];
  if (dpoint) {
    // a point that a 3D wireframe distance names is an entity of A: its increment is part of x
    std::vector<int32_t> jq(d.njp ? d.np : 0, -1);
    if (d.njp) {
      CUDA_OR(p, cudaMemcpyAsync(jq.data(), p->jq, sizeof(int32_t) * d.np, cudaMemcpyDeviceToHost, p->stream));
      CUDA_OR(p, cudaStreamSynchronize(p->stream));
    }
    for (int64_t i = 0; i < d.np; ++i)
      for (int k = 0; k < 3; ++k)
        dpoint[3 * i + k] = (d.njp && jq[i] >= 0) ? x[6 * (d.jbase() + jq[i]) + k] : df[4 * i + k];
  }
  if (dline) for (int64_t i = 0; i < d.nl; ++i) for (int k = 0; k < 4; ++k) dline[4 * i + k] = df[4 * (d.np + i) + k];
  if (pcg_iters) *pcg_iters = p->hS->iters;
  if (pcg_rel) *pcg_rel = p->hS->bnorm2 > 0 ? std::sqrt(p->hS->rr / p->hS->bnorm2) : 0.0;
  if (pred) *pred = p->hS->pred;
  return BA_OK;
}

// ---------------------------------------------------------------------------
// learned preconditioner
extern "C" ba_status ba_precond_set_weights(ba_problem* p, const float* params, int64_t n) {
  if (!p || !params) return BA_ERR_ARG;
  if (n != ba_precond_param_count()) return set_err(p, BA_ERR_ARG, "wrong number of preconditioner parameters");
  ba_status s = freeze(p);
  if (s) return s;
  if ((s = precond_alloc_features(*p))) return set_err(p, s, "device allocation failed");
  if ((s = precond_set_weights(*p, params))) return set_err(p, s, "could not upload the preconditioner weights");
  return BA_OK;
}

extern "C" ba_status ba_precond_features(ba_problem* p, float* X, uint8_t* mask) {
  if (!p) return BA_ERR_ARG;
  if (!p->have_reduced) return set_err(p, BA_ERR_STATE, "no reduced system built (call ba_build_reduced)");
  ba_status s = precond_alloc_features(*p);
  if (s) return set_err(p, s, "device allocation failed");
  if (mixed(p)) launch_pre_features<float>(*p); else launch_pre_features<double>(*p);
  CUDA_OR(p, cudaGetLastError());
  if (X && (s = put_out(p, BA_MEM_HOST, X, (const float*)p->pre_X, 32 * (size_t)p->d.na))) return s;
  if (mask && (s = put_out(p, BA_MEM_HOST, mask, (const uint8_t*)p->pre_mask, (size_t)p->d.na))) return s;
  return BA_OK;
}

extern "C" ba_status ba_precond_blocks(ba_problem* p, double* blocks, int* fallbacks) {
  if (!p || !blocks) return BA_ERR_ARG;
  if (!p->have_reduced) return set_err(p, BA_ERR_STATE, "no reduced system built (call ba_build_reduced)");
  if (p->opt.precond == BA_PRECOND_LEARNED && p->pre_ready) {
    if (mixed(p)) launch_pre_learned<float>(*p); else launch_pre_learned<double>(*p);
  } else {
    if (mixed(p)) launch_precond<float>(*p); else launch_precond<double>(*p);
  }
  CUDA_OR(p, cudaGetLastError());
  const size_t n = (size_t)BS2 * p->d.na;
  ba_status s;
  if (mixed(p)) {
    std::vector<float> h(n);
    if ((s = put_out(p, BA_MEM_HOST, h.data(), (const float*)p->Minv, n))) return s;
    for (size_t i = 0; i < n; ++i) blocks[i] = h[i];
  } else if ((s = put_out(p, BA_MEM_HOST, blocks, (const double*)p->Minv, n))) {
    return s;
  }
  if (fallbacks) {
    *fallbacks = 0;
    if (p->opt.precond == BA_PRECOND_LEARNED && p->pre_ready)
      CUDA_OR(p, cudaMemcpy(fallbacks, p->pre_fallbacks, sizeof(int), cudaMemcpyDeviceToHost));
  }
  return BA_OK;
}

// ---------------------------------------------------------------------------
// batched windows: many independent problems, one persistent launch in a CUDA graph
#include <map>
#include <mutex>

namespace {
struct BatchCfg {
  int threads = 256;
  int per_sm = 1;   // CTAs per SM (windows of one CTA)
  int nct = 1;      // CTAs per window: a thread-block cluster of nct CTAs works on one window
  int nbig = 0;     // with nct > 1: the largest nbig windows run on clusters, the others on single CTAs (-1: all)
};
std::map<std::string, BatchCfg> g_batch_cache;   // (GPU, precision, size class) -> launch shape
std::mutex g_batch_lock;
}  // namespace

template <class T>
static ba_status solve_batch_t(ba_problem* const* w, int n, int iters, ba_solve_report* rep, int autotune) {
  ba_problem* p0 = w[0];
  cudaStream_t st = p0->stream;
  const size_t dsz = window_desc_size<T>();
  std::vector<unsigned char> host(dsz * (size_t)n);
  std::vector<std::pair<int64_t, int>> sz;
  int64_t max_nch = 1, max_work = 1;
  for (int i = 0; i < n; ++i) {
    ba_problem* p = w[i];
    if (!p->win_state) {
      p->win_state = p->dnew<int>(8);
      if (!p->win_state) return set_err(p0, BA_ERR_OOM, "device allocation failed");
    }
    int s0[8] = {p->cur, p->have_lin ? 1 : 0, 0, 0, 0, 0, 0, 0};
    CUDA_OR(p0, cudaMemcpyAsync(p->win_state, s0, sizeof(s0), cudaMemcpyHostToDevice, st));
    CUDA_OR(p0, cudaStreamSynchronize(st));
    fill_window_desc<T>(*p, host.data() + dsz * i);
    int32_t nch = 0;
    CUDA_OR(p0, cudaMemcpy(&nch, p->row_chunk0 + p->d.na, sizeof(int32_t), cudaMemcpyDeviceToHost));
    max_nch = std::max<int64_t>(max_nch, nch);
    const int64_t work = p->d.nr + p->d.nf;
    max_work = std::max(max_work, work);
    sz.push_back({-work, i});
  }
  std::sort(sz.begin(), sz.end());
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = sz[i].second;
  // the batch's identity: its windows (by serial, in order), the iteration count and the precision; a graph
  // kept from an earlier call with the same identity is launched again with its buffers
  std::vector<uint64_t> bkey;
  bkey.push_back((uint64_t)iters);
  bkey.push_back(sizeof(T));
  for (int i = 0; i < n; ++i) bkey.push_back(w[i]->serial);
  auto& bg = p0->bgraph;
  const bool reuse = bg.exec && bg.key == bkey;
  if (!reuse) {
    release_batch_graph(p0);
    bg.desc = p0->alloc.get(host.size());
    bg.order = p0->alloc.get(sizeof(int) * n);
    bg.queue = p0->alloc.get(2 * sizeof(int));
    if (!bg.desc || !bg.order || !bg.queue) { release_batch_graph(p0); return set_err(p0, BA_ERR_OOM, "device allocation failed"); }
  }
  void* d_desc = bg.desc;
  int* d_order = (int*)bg.order;
  int* d_queue = (int*)bg.queue;
  CUDA_OR(p0, cudaMemcpyAsync(d_desc, host.data(), host.size(), cudaMemcpyHostToDevice, st));
  CUDA_OR(p0, cudaMemcpyAsync(d_order, order.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
  const size_t smem = sizeof(double) * 6 * (size_t)max_nch;
  if (smem > 200 * 1024) return set_err(p0, BA_ERR_ARG, "a window's reduced system is too large for the batched kernel");
  int dev = 0, sms = 0;
  CUDA_OR(p0, cudaGetDevice(&dev));
  CUDA_OR(p0, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  cudaDeviceProp prop;
  CUDA_OR(p0, cudaGetDeviceProperties(&prop, dev));
  int cls = 0;
  while ((int64_t(1) << cls) < max_work) ++cls;
  const std::string key = std::string(prop.name) + "/" + (sizeof(T) == 4 ? "f32" : "f64") + "/" + std::to_string(cls);
  BatchCfg cfg;
  bool cached = false;
  const int forced = p0->opt.batch_ctas_per_window;
  if (forced != 0 && forced != 1 && forced != 2 && forced != 4)
    return set_err(p0, BA_ERR_ARG, "batch_ctas_per_window must be 0, 1, 2 or 4");
  if (forced > 0) {
    cfg.nct = forced;
    cfg.nbig = -1;
    cached = true;
    if (forced > 1 && window_clusters<T>(cfg.threads, smem, forced) < 1)
      return set_err(p0, BA_ERR_ARG, "no cluster of that many window CTAs fits this GPU");
  } else {
    std::lock_guard<std::mutex> g(g_batch_lock);
    auto it = g_batch_cache.find(key);
    if (it != g_batch_cache.end()) { cfg = it->second; cached = true; }
  }
  auto grid_of = [&](const BatchCfg& c) {
    if (c.nct > 1) {
      const int ncl = window_clusters<T>(c.threads, smem, c.nct);
      return std::max(1, std::min(n, ncl)) * c.nct;
    }
    int occ = windows_per_sm<T>(c.threads, smem);
    return std::max(1, std::min(n, sms * std::max(1, std::min(occ, c.per_sm))));
  };
  // ---- autotuner: time one LM step of every candidate shape from the same state (scalars and per-window
  // state are restored after each trial; the parameters a trial may change are the candidate set only)
  if (autotune && !cached) {
    std::vector<DevScalars> snapS(n);
    std::vector<std::array<int, 5>> snapW(n);
    for (int i = 0; i < n; ++i) {
      CUDA_OR(p0, cudaMemcpy(&snapS[i], w[i]->S, sizeof(DevScalars), cudaMemcpyDeviceToHost));
      CUDA_OR(p0, cudaMemcpy(snapW[i].data(), w[i]->win_state, sizeof(int) * 5, cudaMemcpyDeviceToHost));
    }
    // launch shapes: threads per CTA, CTAs per SM, and CTAs per window (a cluster splits a window's features,
    // Schur units and reduced-system rows over its CTAs: the largest windows otherwise set the makespan)
    const BatchCfg cands[] = {{128, 1, 1, 0}, {128, 2, 1, 0}, {256, 1, 1, 0}, {256, 2, 1, 0}, {256, 1, 2, -1},
                              {256, 1, 2, 32}, {256, 1, 4, 16},   {256, 1, 4, 32},  {256, 1, 4, 64}};
    float best = 1e30f;
    cudaEvent_t e0, e1;
    CUDA_OR(p0, cudaEventCreate(&e0));
    CUDA_OR(p0, cudaEventCreate(&e1));
    for (const BatchCfg& c : cands) {
      if (c.per_sm > 1 && windows_per_sm<T>(c.threads, smem) < c.per_sm) continue;
      if (c.nct > 1 && window_clusters<T>(c.threads, smem, c.nct) < 1) continue;
      CUDA_OR(p0, cudaEventRecord(e0, st));
      CUDA_OR(p0, launch_windows<T>(st, d_desc, d_order, n, c.nbig < 0 ? n : std::min(n, c.nbig), 1, d_queue,
                                    c.threads, grid_of(c), smem, c.nct));
      CUDA_OR(p0, cudaEventRecord(e1, st));
      CUDA_OR(p0, cudaEventSynchronize(e1));
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) { best = ms; cfg = c; }
      for (int i = 0; i < n; ++i) {
        CUDA_OR(p0, cudaMemcpy(w[i]->S, &snapS[i], sizeof(DevScalars), cudaMemcpyHostToDevice));
        CUDA_OR(p0, cudaMemcpy(w[i]->win_state, snapW[i].data(), sizeof(int) * 5, cudaMemcpyHostToDevice));
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::lock_guard<std::mutex> g(g_batch_lock);
    g_batch_cache[key] = cfg;
  }
  // ---- the solve: queue reset + persistent kernel, captured once in a graph (kept for the next call with
  // the same batch) and launched.  Capture is not allowed on the legacy default stream: capture and launch on a
  // private stream that starts after the caller's stream has drained
  const int grid = grid_of(cfg);
  CUDA_OR(p0, cudaStreamSynchronize(st));
  if (!reuse || bg.threads != cfg.threads || bg.grid != grid || bg.nct != cfg.nct || bg.nbig != cfg.nbig) {
    if (bg.exec) { cudaGraphExecDestroy(bg.exec); bg.exec = nullptr; }
    if (bg.graph) { cudaGraphDestroy(bg.graph); bg.graph = nullptr; }
    if (!bg.stream) CUDA_OR(p0, cudaStreamCreateWithFlags(&bg.stream, cudaStreamNonBlocking));
    CUDA_OR(p0, cudaStreamBeginCapture(bg.stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t le = launch_windows<T>(bg.stream, d_desc, d_order, n, cfg.nbig < 0 ? n : std::min(n, cfg.nbig), iters,
                                       d_queue, cfg.threads, grid, smem, cfg.nct);
    cudaError_t ce = cudaStreamEndCapture(bg.stream, &bg.graph);
    if (le != cudaSuccess || ce != cudaSuccess) {
      cudaGetLastError();
      release_batch_graph(p0);
      return set_err(p0, BA_ERR_CUDA, std::string("batched graph capture: ") + cudaGetErrorString(le != cudaSuccess ? le : ce));
    }
    CUDA_OR(p0, cudaGraphInstantiate(&bg.exec, bg.graph, 0));
    bg.key = bkey;
    bg.threads = cfg.threads;
    bg.grid = grid;
    bg.nct = cfg.nct;
    bg.nbig = cfg.nbig;
  }
  cudaEvent_t e0, e1;
  CUDA_OR(p0, cudaEventCreate(&e0));
  CUDA_OR(p0, cudaEventCreate(&e1));
  CUDA_OR(p0, cudaEventRecord(e0, bg.stream));
  CUDA_OR(p0, cudaGraphLaunch(bg.exec, bg.stream));
  CUDA_OR(p0, cudaEventRecord(e1, bg.stream));
  CUDA_OR(p0, cudaEventSynchronize(e1));
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CUDA_OR(p0, cudaGetLastError());
  p0->batch_threads = cfg.threads;
  p0->batch_nct = cfg.nct;
  p0->batch_nbig = cfg.nct > 1 ? (cfg.nbig < 0 ? n : std::min(n, cfg.nbig)) : 0;
  p0->batch_grid = grid;
  // ---- bring every window's host state up to date
  for (int i = 0; i < n; ++i) {
    ba_problem* p = w[i];
    int sw[8];
    CUDA_OR(p0, cudaMemcpy(sw, p->win_state, sizeof(sw), cudaMemcpyDeviceToHost));
    unsigned long long wns = 0;
    std::memcpy(&wns, sw + 6, sizeof(wns));
    CUDA_OR(p0, cudaMemcpy(p->hS, p->S, sizeof(DevScalars), cudaMemcpyDeviceToHost));
    p->cur = sw[0];
    p->have_lin = sw[1] != 0;
    p->have_reduced = false;
    if (rep) {
      ba_solve_report& r = rep[i];
      std::memset(&r, 0, sizeof(r));
      r.iters = sw[2];
      r.accepted_steps = sw[3];
      r.converged = sw[4] > 0;
      r.cost = p->hS->E;
      r.cost_px = p->hS->Epx;
      r.ms_total = ms;
      r.ms_window = (double)wns * 1e-6;
    }
  }
  return BA_OK;
}

extern "C" ba_status ba_solve_batch(ba_problem* const* windows, int n, int lm_iters, int autotune,
                                    ba_solve_report* reports) {
  if (!windows || n <= 0 || lm_iters <= 0) return BA_ERR_ARG;
  for (int i = 0; i < n; ++i)
    if (!windows[i]) return BA_ERR_ARG;
  ba_problem* p0 = windows[0];
  for (int i = 0; i < n; ++i) {
    ba_problem* p = windows[i];
    if (p->opt.precision != p0->opt.precision)
      return set_err(p0, BA_ERR_ARG, "all windows of a batch must use the same precision");
    if (p->device != p0->device) return set_err(p0, BA_ERR_ARG, "all windows of a batch must be on one device");
    ba_status s = freeze(p);
    if (!s && p->nrel) s = set_err(p, BA_ERR_ARG, "inter-group relations are not supported in batched windows");
    if (!s && p->d.nk) s = set_err(p, BA_ERR_ARG, "refined intrinsics (cam_dof 9) are not supported in batched windows");
    if (!s && p->d.njp) s = set_err(p, BA_ERR_ARG, "3D wireframe distances are not supported in batched windows");
    if (!s && (p->d.ngs() || p->d.nbx()))
      s = set_err(p, BA_ERR_ARG, "spheres, cylinders, cones, ellipsoids and cuboids are not supported in batched windows");
    if (!s) s = ensure_sstore(p, true);
    if (s) return set_err(p0, s, "window " + std::to_string(i) + ": " + p->err);
    if (p->typed)
      return set_err(p0, BA_ERR_STATE, "window " + std::to_string(i) +
                                           ": a problem already stepped on its own cannot join a batch (its reduced "
                                           "system has the typed storage of the grid path)");
    if (reports) reports[i].cost0 = p->hS->E;
  }
  std::vector<double> c0(n);
  for (int i = 0; i < n; ++i) c0[i] = windows[i]->hS->E;
  ba_status s = mixed(p0) ? solve_batch_t<float>(windows, n, lm_iters, reports, autotune)
                          : solve_batch_t<double>(windows, n, lm_iters, reports, autotune);
  if (s == BA_OK && reports)
    for (int i = 0; i < n; ++i) reports[i].cost0 = c0[i];
  return s;
}

extern "C" ba_status ba_batch_ctas_per_window(const ba_problem* p, int* ctas, int* windows_on_clusters) {
  if (!p) return BA_ERR_ARG;
  if (ctas) *ctas = p->batch_nct;
  if (windows_on_clusters) *windows_on_clusters = p->batch_nbig;
  return BA_OK;
}

extern "C" ba_status ba_batch_launch_shape(const ba_problem* p, int* threads, int* grid) {
  if (!p) return BA_ERR_ARG;
  if (threads) *threads = p->batch_threads;
  if (grid) *grid = p->batch_grid;
  return BA_OK;
}
