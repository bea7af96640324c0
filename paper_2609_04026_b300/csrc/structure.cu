// One-time structure build (K0): the analogue of a sparse solver's symbolic
// analysis, which the paper observes only on the first iteration of each BA
// call (Section 4, Fig. 3c).  It runs on the GPU from the residual records
// that ba_add_observations copied there:
//   * every record is validated (an out of range id or a non-finite measurement
//     gives BA_ERR_ARG naming the first bad record) and merged in input order,
//   * the residual records are ordered feature-major (each residual touches
//     exactly one feature, Section 3.2-3.4, so H_ff is block-diagonal), and by
//     camera inside a feature, with a stable LSD radix sort,
//   * every (feature, kept entity) pair gets a "slot" that will hold its W
//     block and its direct contribution to H_aa,
//   * the block pattern of S over A = cameras u groups (every pair of entities
//     that share a feature, Section 3.3 sparsity analysis) is marked in a
//     symmetric bitmap of A x A and read out as full block-CSR (both triangles,
//     for the SpMV), padded and interleaved for coalesced loads,
//   * for every upper block of S the slot pairs (e_a, e_b) whose product
//     W_a V^-1 W_b^T lands in it are listed in feature order (a stable radix
//     sort of the pairs by block) and cut into work units of at most UNIT_MAX
//     pairs, so that the Schur kernels accumulate each block in a fixed order
//     without atomics.
// Every step is deterministic: the same input gives the same structure, and the
// orders are those of a sequential build (features ascending, cameras ascending
// inside a feature, input order among equal keys).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "ba_internal.cuh"

namespace ba {

static constexpr int UNIT_MAX = 1024;     // pairs per Schur work unit
static constexpr int UNIT_LONG = 128;     // units with more pairs are scheduled first
static constexpr int PACK_MAX = 32;       // pairs of a pack of small units (one per lane)

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

// ---------------------------------------------------------------------------
// temporary device memory of the build, released when the build returns
struct Scratch {
  Alloc* al;
  cudaStream_t st;
  std::vector<void*> ptrs;
  Scratch(Alloc* a, cudaStream_t s) : al(a), st(s) {}
  ~Scratch() {
    cudaStreamSynchronize(st);   // kernels of a build that stopped early may still read these buffers
    for (void* p : ptrs) al->put(p);
  }
  template <class X>
  X* get(int64_t n) {
    void* p = al->get(sizeof(X) * (size_t)(n > 0 ? n : 1));
    if (p) ptrs.push_back(p);
    return (X*)p;
  }
};

static inline unsigned grid_of(int64_t n, int nt) { return (unsigned)std::max<int64_t>(1, (n + nt - 1) / nt); }
static inline int bits_for(int64_t n) {   // bits to hold values in [0, n)
  int b = 0;
  while (b < 62 && ((int64_t)1 << b) < n) ++b;
  return b;
}

// ---------------------------------------------------------------------------
// exclusive scan of int64 values (three phases: tile sums, scan of the tile sums, tile scans)
constexpr int SC_NT = 256, SC_ITEMS = 8, SC_TILE = SC_NT * SC_ITEMS;

__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t* sh, int64_t* total) {
  // sh: SC_NT / 32 + 1 entries
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[w] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t s = 0;
    for (int i = 0; i < SC_NT / 32; ++i) { const int64_t c = sh[i]; sh[i] = s; s += c; }
    sh[SC_NT / 32] = s;
  }
  __syncthreads();
  const int64_t r = x - v + sh[w];
  *total = sh[SC_NT / 32];
  __syncthreads();
  return r;
}

__global__ void k_scan_tiles(const int64_t* __restrict__ in, int64_t n, int64_t* __restrict__ tsum) {
  __shared__ int64_t sh[SC_NT / 32 + 1];
  const int64_t base = blockIdx.x * (int64_t)SC_TILE + (int64_t)threadIdx.x * SC_ITEMS;
  int64_t s = 0;
#pragma unroll
  for (int i = 0; i < SC_ITEMS; ++i) s += (base + i < n) ? in[base + i] : 0;
  int64_t tot;
  block_excl_scan(s, sh, &tot);
  if (threadIdx.x == 0) tsum[blockIdx.x] = tot;
}

__global__ void k_scan_apply(const int64_t* __restrict__ in, int64_t n, const int64_t* __restrict__ toff,
                             int64_t* __restrict__ out) {
  __shared__ int64_t sh[SC_NT / 32 + 1];
  const int64_t base = blockIdx.x * (int64_t)SC_TILE + (int64_t)threadIdx.x * SC_ITEMS;
  int64_t v[SC_ITEMS], s = 0;
#pragma unroll
  for (int i = 0; i < SC_ITEMS; ++i) { v[i] = (base + i < n) ? in[base + i] : 0; s += v[i]; }
  int64_t tot;
  int64_t run = block_excl_scan(s, sh, &tot) + toff[blockIdx.x];
#pragma unroll
  for (int i = 0; i < SC_ITEMS; ++i) {
    if (base + i < n) out[base + i] = run;
    run += v[i];
  }
}

// out[i] = sum of in[0..i) for i in [0, n], out has n + 1 entries (in and out may alias only if n == 0)
static ba_status scan_excl(Problem& P, Scratch& S, const int64_t* in, int64_t* out, int64_t n) {
  if (n == 0) {
    CU(cudaMemsetAsync(out, 0, sizeof(int64_t), P.stream));
    return BA_OK;
  }
  const int64_t nt = (n + SC_TILE - 1) / SC_TILE;
  int64_t* tsum = S.get<int64_t>(nt);
  int64_t* toff = S.get<int64_t>(nt + 1);
  if (!tsum || !toff) return fail(P, BA_ERR_OOM, "device allocation failed");
  k_scan_tiles<<<(unsigned)nt, SC_NT, 0, P.stream>>>(in, n, tsum);
  if (nt == 1) {
    CU(cudaMemsetAsync(toff, 0, sizeof(int64_t), P.stream));
    CU(cudaMemcpyAsync(toff + 1, tsum, sizeof(int64_t), cudaMemcpyDeviceToDevice, P.stream));
  } else {
    ba_status s = scan_excl(P, S, tsum, toff, nt);
    if (s) return s;
  }
  k_scan_apply<<<(unsigned)nt, SC_NT, 0, P.stream>>>(in, n, toff, out);
  CU(cudaMemcpyAsync(out + n, toff + nt, sizeof(int64_t), cudaMemcpyDeviceToDevice, P.stream));   // the total
  CU(cudaGetLastError());
  return BA_OK;
}

// ---------------------------------------------------------------------------
// stable LSD radix sort of (key, value) u32 pairs by the low `bits` bits of the key, 8 bits per pass.
// A tile of RS_TILE keys is split into per-warp runs of consecutive keys; inside a warp the rank of a
// key among equal digits comes from __match_any_sync, so the scatter keeps the input order of equal
// digits (stability) without any atomics on global memory.
constexpr int RS_NT = 256, RS_ITEMS = 16, RS_TILE = RS_NT * RS_ITEMS, RS_NW = RS_NT / 32;

__global__ void k_rs_hist(const uint32_t* __restrict__ keys, int64_t n, int shift, int64_t* __restrict__ hist,
                          int64_t ntiles) {
  __shared__ unsigned h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = blockIdx.x * (int64_t)RS_TILE;
  for (int i = threadIdx.x; i < RS_TILE; i += RS_NT) {
    const int64_t k = base + i;
    if (k < n) atomicAdd(&h[(keys[k] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(RS_NT) k_rs_scatter(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                                                      uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, int64_t n,
                                                      int shift, const int64_t* __restrict__ off, int64_t ntiles) {
  __shared__ unsigned wcnt[RS_NW][256];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < RS_NW * 256; i += RS_NT) (&wcnt[0][0])[i] = 0;
  __syncthreads();
  const int64_t base = blockIdx.x * (int64_t)RS_TILE + (int64_t)warp * 32 * RS_ITEMS;
  uint32_t k[RS_ITEMS], v[RS_ITEMS], loc[RS_ITEMS];
#pragma unroll
  for (int it = 0; it < RS_ITEMS; ++it) {
    const int64_t idx = base + it * 32 + lane;
    const bool ok = idx < n;
    k[it] = ok ? kin[idx] : 0u;
    v[it] = ok ? vin[idx] : 0u;
    const unsigned d = (k[it] >> shift) & 255u;
    const unsigned peers = __match_any_sync(0xffffffffu, ok ? d : 0x100u + lane);
    const unsigned rank = __popc(peers & ((1u << lane) - 1u));
    const unsigned before = ok ? wcnt[warp][d] : 0u;
    __syncwarp();
    if (ok && rank == 0) wcnt[warp][d] = before + __popc(peers);
    __syncwarp();
    loc[it] = before + rank;
  }
  __syncthreads();
  // exclusive prefix of the per-warp counts of each digit (warps hold consecutive runs of the tile)
  for (int d = threadIdx.x; d < 256; d += RS_NT) {
    unsigned s = 0;
#pragma unroll
    for (int w = 0; w < RS_NW; ++w) { const unsigned c = wcnt[w][d]; wcnt[w][d] = s; s += c; }
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < RS_ITEMS; ++it) {
    const int64_t idx = base + it * 32 + lane;
    if (idx < n) {
      const unsigned d = (k[it] >> shift) & 255u;
      const int64_t dst = off[(int64_t)d * ntiles + blockIdx.x] + wcnt[warp][d] + loc[it];
      kout[dst] = k[it];
      vout[dst] = v[it];
    }
  }
}

// sorts (k, v) in place (k and v end up holding the sorted pairs); k2 / v2 are work buffers of n entries
static ba_status radix_sort(Problem& P, Scratch& S, uint32_t* k, uint32_t* v, uint32_t* k2, uint32_t* v2, int64_t n,
                            int bits) {
  if (n <= 1 || bits <= 0) return BA_OK;
  const int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
  int64_t* hist = S.get<int64_t>(256 * ntiles);
  int64_t* off = S.get<int64_t>(256 * ntiles + 1);
  if (!hist || !off) return fail(P, BA_ERR_OOM, "device allocation failed");
  uint32_t *ka = k, *va = v, *kb = k2, *vb = v2;
  for (int shift = 0; shift < bits; shift += 8) {
    k_rs_hist<<<(unsigned)ntiles, RS_NT, 0, P.stream>>>(ka, n, shift, hist, ntiles);
    ba_status s = scan_excl(P, S, hist, off, 256 * ntiles);
    if (s) return s;
    k_rs_scatter<<<(unsigned)ntiles, RS_NT, 0, P.stream>>>(ka, va, kb, vb, n, shift, off, ntiles);
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  if (ka != k) {
    CU(cudaMemcpyAsync(k, ka, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, P.stream));
    CU(cudaMemcpyAsync(v, va, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, P.stream));
  }
  CU(cudaGetLastError());
  return BA_OK;
}

// ---------------------------------------------------------------------------
// build kernels
__global__ void k_iota_key(const int32_t* __restrict__ src, int64_t n, int add, uint32_t* __restrict__ key,
                           uint32_t* __restrict__ val) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) { key[i] = (uint32_t)(src[i] + add); val[i] = (uint32_t)i; }
}

// key[j] = feature of residual val[j] (the permutation sorted by camera so far)
__global__ void k_gather_key(const int32_t* __restrict__ feat, const uint32_t* __restrict__ val, int64_t n,
                             uint32_t* __restrict__ key) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j < n) key[j] = (uint32_t)feat[val[j]];
}

__global__ void k_count(const int32_t* __restrict__ id, int64_t n, unsigned long long* __restrict__ cnt) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j < n) atomicAdd(&cnt[id[j]], 1ull);
}

__global__ void k_i64_to_i32(const int64_t* __restrict__ a, int64_t n, int32_t* __restrict__ b) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j < n) b[j] = (int32_t)a[j];
}

// the points that a 3D wireframe distance names (mark[p] = 1), their ranks (ascending point id) and the
// feature key of every record: a named point's residuals are a zero-dimension feature after the points and
// lines (nf_real + rank); the records themselves keep the point id
__global__ void k_mark_jpt(const int8_t* __restrict__ kind, const int32_t* __restrict__ grp, int64_t n,
                           int64_t* __restrict__ mark) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j < n && kind[j] == R_WF3D) mark[grp[j]] = 1;   // every writer stores the same value
}
__global__ void k_jq(const int64_t* __restrict__ mark, const int64_t* __restrict__ rank, int64_t np,
                     int32_t* __restrict__ jq, int32_t* __restrict__ jp_pt) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= np) return;
  jq[p] = mark[p] ? (int32_t)rank[p] : -1;
  if (mark[p]) jp_pt[rank[p]] = (int32_t)p;
}
__global__ void k_fkey(const int32_t* __restrict__ feat, const int32_t* __restrict__ jq, int64_t np, int64_t nf_real,
                       int64_t n, int32_t* __restrict__ fkey) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int32_t f = feat[j];
  fkey[j] = (f < np && jq[f] >= 0) ? (int32_t)(nf_real + jq[f]) : f;
}

struct SlotArgs {
  const int32_t *order, *fres_off, *cam, *grp;
  const int8_t* kind;
  const uint8_t* fixed;
  int64_t nf, nc, npl;
  int* err;   // bit 0: two planes on one feature, bit 1: two VPs on one line
  const int32_t* cam_k;   // refined intrinsics: per camera its intrinsics entity (else null)
  int64_t kbase;          // A index of intrinsics entity 0
  int64_t sbase, nsp, ncy;   // A index of the first sphere; spheres, cylinders (cones follow)
  int64_t bbase, nel, ncu;   // A index of the first ellipsoid entity; ellipsoids, cuboids
  const int32_t* jq;         // per point its index among the wireframe-coupled points (or -1), or null
  int64_t jbase, nf_real;    // A index of the first wireframe-coupled point; points and lines
};

// the positional group of residual record i as an A index (plane, sphere, cylinder, cone), or -1
__device__ __forceinline__ int64_t pos_group(const SlotArgs& a, int k, int32_t g) {
  if (k == R_PLANE_POINT || k == R_PLANE_LINE || k == R_PLANE_POINT3 || k == R_PLANE_LINE3) return a.nc + g;
  if (k == R_SPHERE_POINT) return a.sbase + g;
  if (k == R_CYL_POINT) return a.sbase + a.nsp + g;
  if (k == R_CONE_POINT) return a.sbase + a.nsp + a.ncy + g;
  if (k == R_ELL_POINT) return a.bbase + g;
  if (k == R_CUB_POINT || k == R_CUB_LINE) return a.bbase + 2 * a.nel + g;
  return -1;
}
// a 9-parameter group's second entity (A index), or -1
__device__ __forceinline__ int64_t pos_group2(const SlotArgs& a, int k, int32_t g) {
  if (k == R_ELL_POINT) return a.bbase + a.nel + g;
  if (k == R_CUB_POINT || k == R_CUB_LINE) return a.bbase + 2 * a.nel + a.ncu + g;
  return -1;
}
__device__ __forceinline__ uint8_t pos_type(const SlotArgs& a, int64_t e) {
  return e < a.sbase ? ENT_PLANE : e < a.sbase + a.nsp ? ENT_SPHERE : e < a.sbase + a.nsp + a.ncy ? ENT_CYL
       : e < a.bbase ? ENT_CONE : e < a.bbase + a.nel ? ENT_ELL1 : e < a.bbase + 2 * a.nel ? ENT_ELL2
       : e < a.bbase + 2 * a.nel + a.ncu ? ENT_CUB1 : ENT_CUB2;
}

// the extra 3-dimension entity (A index) that residual j of feature f names besides its camera and groups, or
// -1: its camera's intrinsics entity (refined intrinsics); the point of a 3D wireframe distance (a line's
// residual); the point itself for a residual of a wireframe-coupled point (a zero-dimension feature)
__device__ __forceinline__ int64_t slot_extra(const SlotArgs& a, int64_t f, int32_t j) {
  const int32_t i = a.order[j];
  if (a.cam_k) {
    const int c = a.cam[i];
    return c >= 0 ? a.kbase + a.cam_k[c] : -1;
  }
  if (a.jq) {
    if (f >= a.nf_real) return a.jbase + (f - a.nf_real);
    if (a.kind[i] == R_WF3D) return a.jbase + a.jq[a.grp[i]];
  }
  return -1;
}

// distinct kept entities of a feature (cameras ascending, then its plane, then its VP, then the intrinsics
// entities of its cameras or its wireframe-coupled points, ascending)
__global__ void k_slot_count(SlotArgs a, int64_t* __restrict__ nslot) {
  const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= a.nf) return;
  int n = 0, prev = -1, vp = -1;
  int64_t plane = -1, second = -1;   // the positional group (A index) and a 9-parameter group's second entity
  const int32_t r0 = a.fres_off[f], r1 = a.fres_off[f + 1];
  for (int32_t j = r0; j < r1; ++j) {
    const int32_t i = a.order[j];
    const int c = a.cam[i];
    if (c >= 0 && a.fixed[c] != 0x3F && c != prev) { ++n; prev = c; }
    const int k = a.kind[i];
    const int64_t pg = pos_group(a, k, a.grp[i]);
    if (pg >= 0) {
      if (plane >= 0 && plane != pg) atomicOr(a.err, 1);
      plane = pg;
      second = pos_group2(a, k, a.grp[i]);
    } else if (k == R_VP) {
      if (vp >= 0 && vp != a.grp[i]) atomicOr(a.err, 2);
      vp = a.grp[i];
    }
    // an extra entity counts at the first residual that names it
    const int64_t kk = slot_extra(a, f, j);
    if (kk >= 0) {
      bool seen = false;
      for (int32_t j2 = r0; j2 < j && !seen; ++j2) seen = slot_extra(a, f, j2) == kk;
      n += seen ? 0 : 1;
    }
  }
  nslot[f] = n + (plane >= 0) + (second >= 0) + (vp >= 0);
}

struct SlotFill {
  int32_t *fslot_off, *slot_ent, *slot_feat, *feat_plane_slot, *rslot_c, *rslot_g, *rslot_k;
  uint8_t* slot_type;
};

__global__ void k_slot_fill(SlotArgs a, const int64_t* __restrict__ soff, SlotFill o) {
  const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f > a.nf) return;
  o.fslot_off[f] = (int32_t)soff[f];
  if (f == a.nf) return;
  const int32_t r0 = a.fres_off[f], r1 = a.fres_off[f + 1];
  int32_t e = (int32_t)soff[f];
  int prev = -1, vp = -1;
  int64_t plane = -1, second = -1;   // the positional group (A index) and a 9-parameter group's second entity
  for (int32_t j = r0; j < r1; ++j) {
    const int32_t i = a.order[j];
    const int c = a.cam[i];
    const int k = a.kind[i];
    const int64_t pg = pos_group(a, k, a.grp[i]);
    if (pg >= 0) { plane = pg; second = pos_group2(a, k, a.grp[i]); }
    if (k == R_VP) vp = a.grp[i];
    if (c >= 0 && a.fixed[c] != 0x3F) {
      if (c != prev) {
        o.slot_ent[e] = c;
        o.slot_feat[e] = (int32_t)f;
        o.slot_type[e] = ENT_CAM;
        prev = c;
        ++e;
      }
      o.rslot_c[j] = e - 1;
    } else {
      o.rslot_c[j] = -1;
    }
  }
  const int32_t plane_slot = plane >= 0 ? e : -1;
  if (plane >= 0) {
    o.slot_ent[e] = (int32_t)plane;
    o.slot_feat[e] = (int32_t)f;
    o.slot_type[e] = pos_type(a, plane);
    ++e;
  }
  if (second >= 0) {   // right after the first entity's slot (points have no VP slot)
    o.slot_ent[e] = (int32_t)second;
    o.slot_feat[e] = (int32_t)f;
    o.slot_type[e] = pos_type(a, second);
    ++e;
  }
  const int32_t vp_slot = vp >= 0 ? e : -1;
  if (vp >= 0) {
    o.slot_ent[e] = (int32_t)(a.nc + a.npl + vp);
    o.slot_feat[e] = (int32_t)f;
    o.slot_type[e] = ENT_VP;
    ++e;
  }
  o.feat_plane_slot[f] = plane_slot;
  for (int32_t j = r0; j < r1; ++j) {
    const int k = a.kind[a.order[j]];
    const bool on_plane = pos_group(a, k, 0) >= 0;
    o.rslot_g[j] = on_plane ? plane_slot : (k == R_VP ? vp_slot : -1);
  }
  if (!a.cam_k && !a.jq) return;
  // the extra entities (intrinsics of the feature's cameras, or wireframe-coupled points) in ascending order
  // (the slots of a feature are in entity order), then every residual's slot among them
  const int32_t k0 = e;
  int64_t last = -1;
  for (;;) {
    int64_t nxt = INT64_MAX;
    for (int32_t j = r0; j < r1; ++j) {
      const int64_t kk = slot_extra(a, f, j);
      if (kk > last && kk < nxt) nxt = kk;
    }
    if (nxt == INT64_MAX) break;
    o.slot_ent[e] = (int32_t)nxt;
    o.slot_feat[e] = (int32_t)f;
    o.slot_type[e] = nxt >= a.jbase ? ENT_JPT : ENT_INTR;
    ++e;
    last = nxt;
  }
  for (int32_t j = r0; j < r1; ++j) {
    const int64_t kk = slot_extra(a, f, j);
    int32_t sk = -1;
    for (int32_t q = k0; q < e && kk >= 0; ++q)
      if (o.slot_ent[q] == (int32_t)kk) { sk = q; break; }
    o.rslot_k[j] = sk;
  }
}

// symmetric bitmap of the block pattern of S: bit (a, b) set when a and b share a feature or a == b
struct Bitmap {
  uint32_t* w;
  int64_t wpr;   // 32-bit words per row
  __device__ __forceinline__ void set(int64_t a, int64_t b) const {
    uint32_t* p = w + a * wpr + (b >> 5);
    const uint32_t bit = 1u << (b & 31);
    if (!(*(volatile uint32_t*)p & bit)) atomicOr(p, bit);
  }
};

__global__ void k_pattern_pairs(const int32_t* __restrict__ fslot_off, const int32_t* __restrict__ slot_ent, int64_t nf,
                                Bitmap bm) {
  const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= nf) return;
  const int32_t s0 = fslot_off[f], s1 = fslot_off[f + 1];
  for (int32_t i = s0; i < s1; ++i) {
    const int64_t a = slot_ent[i];
    for (int32_t j = i + 1; j < s1; ++j) {
      const int64_t b = slot_ent[j];
      bm.set(a, b);
      bm.set(b, a);
    }
  }
}

// inter-group relations couple their two groups directly (H_gg)
__global__ void k_pattern_rel(int64_t n, const int32_t* __restrict__ ga, const int32_t* __restrict__ gb, Bitmap bm) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) { bm.set(ga[i], gb[i]); bm.set(gb[i], ga[i]); }
}

__global__ void k_pattern_diag(int64_t na, Bitmap bm) {
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a < na) bm.set(a, a);
}

// per row: stored blocks, blocks left of the diagonal, and the exclusive popcount prefix of every word
__global__ void k_pattern_rows(int64_t na, Bitmap bm, int32_t* __restrict__ wpre, int64_t* __restrict__ full_cnt,
                               int64_t* __restrict__ pad_cnt, int64_t* __restrict__ up_cnt, int32_t* __restrict__ nlow) {
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= na) return;
  const uint32_t* row = bm.w + a * bm.wpr;
  int32_t* pre = wpre + a * bm.wpr;
  int32_t s = 0;
  for (int64_t w = 0; w < bm.wpr; ++w) {
    pre[w] = s;
    s += __popc(row[w]);
  }
  const int32_t low = pre[a >> 5] + __popc(row[a >> 5] & ((1u << (a & 31)) - 1u));
  full_cnt[a] = s;
  pad_cnt[a] = ((s + 31) / 32) * 32;
  up_cnt[a] = s - low;
  nlow[a] = low;
}

__device__ __forceinline__ int32_t bm_rank(const Bitmap& bm, const int32_t* wpre, int64_t a, int64_t c) {
  const int64_t w = c >> 5;
  return wpre[a * bm.wpr + w] + __popc(bm.w[a * bm.wpr + w] & ((1u << (c & 31)) - 1u));
}

struct RowFill {
  const int64_t *prow, *uptr;
  const int32_t *wpre, *nlow;
  int32_t *pcol, *up_row, *up_full, *up_mirror, *prow32, *row_len;
  const int64_t* full_cnt;
};

__global__ void k_pattern_fill(int64_t na, Bitmap bm, RowFill o) {
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a > na) return;
  o.prow32[a] = (int32_t)o.prow[a];
  if (a == na) return;
  o.row_len[a] = (int32_t)o.full_cnt[a];
  const uint32_t* row = bm.w + a * bm.wpr;
  const int64_t p0 = o.prow[a];
  int32_t k = 0;
  for (int64_t w = 0; w < bm.wpr; ++w) {
    uint32_t bits = row[w];
    while (bits) {
      const int t = __ffs(bits) - 1;
      bits &= bits - 1u;
      const int64_t c = w * 32 + t;
      o.pcol[p0 + k] = (int32_t)c;
      if (c >= a) {
        const int64_t u = o.uptr[a] + (k - o.nlow[a]);
        o.up_row[u] = (int32_t)a;
        o.up_full[u] = (int32_t)(p0 + k);
        o.up_mirror[u] = (int32_t)(o.prow[c] + bm_rank(bm, o.wpre, c, a));
      }
      ++k;
    }
  }
  for (int64_t q = p0 + k; q < o.prow[a + 1]; ++q) o.pcol[q] = (int32_t)a;   // padding: col = row, zero values
}

__global__ void k_pair_count(const int32_t* __restrict__ fslot_off, int64_t nf, int64_t* __restrict__ npf) {
  const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= nf) return;
  const int64_t n = fslot_off[f + 1] - fslot_off[f];
  npf[f] = n * (n + 1) / 2;
}

struct PairGen {
  const int32_t *fslot_off, *slot_ent, *wpre, *nlow;
  const uint8_t* slot_type;
  const int32_t* cam_k;   // refined intrinsics: per camera its entity (else null)
  int64_t kbase;
  int64_t nf_real;        // points and lines; later features are zero-dimension ones
  const int64_t *poff, *uptr;
  Bitmap bm;
  int64_t nf;
  uint32_t *key, *val;
  int32_t *gi, *gj;
  unsigned long long* ucnt;
};

// the pairs of every feature in (i, j >= i) order: key = upper block of S the product lands in
__global__ void k_pair_gen(PairGen g) {
  const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= g.nf) return;
  const int32_t s0 = g.fslot_off[f], s1 = g.fslot_off[f + 1];
  int64_t q = g.poff[f];
  for (int32_t i = s0; i < s1; ++i) {
    const int64_t a = g.slot_ent[i];
    for (int32_t j = i; j < s1; ++j, ++q) {
      const int64_t b = g.slot_ent[j];
      const int64_t u = g.uptr[a] + (bm_rank(g.bm, g.wpre, a, b) - g.nlow[a]);
      g.key[q] = (uint32_t)u;
      g.val[q] = (uint32_t)q;
      g.gi[q] = i;
      // bits 30-31: the direct block of the pair's two entities that the feature's residuals add (camera-plane;
      // camera and its own intrinsics entity; plane-intrinsics)
      uint32_t code = 0;
      if (i != j) {
        const int ti = g.slot_type[i], tj = g.slot_type[j];
        if (ti == ENT_CAM && tj == ENT_PLANE) code = PAIR_CP;
        else if (tj == ENT_JPT) {
          // a wireframe-coupled point: direct blocks with the camera and plane of its own residuals only
          if (f >= g.nf_real) code = ti == ENT_CAM ? PAIR_CK : ti == ENT_PLANE ? PAIR_PK : 0u;
        }
        else if (ti == ENT_CAM && tj == ENT_INTR && g.cam_k && g.kbase + g.cam_k[a] == b) code = PAIR_CK;
        else if (ti == ENT_PLANE && tj == ENT_INTR) code = PAIR_PK;
        else if (ti == ENT_CAM && ent_second(tj)) code = PAIR_CK;
        else if (ti == ENT_CAM && ent_surface(tj)) code = PAIR_CS;
        else if ((ti == ENT_ELL1 && tj == ENT_ELL2) || (ti == ENT_CUB1 && tj == ENT_CUB2)) code = PAIR_G12;
      }
      g.gj[q] = (int32_t)((uint32_t)j | (code << PAIR_SHIFT));
      atomicAdd(&g.ucnt[u], 1ull);
    }
  }
}

__global__ void k_pair_place(const uint32_t* __restrict__ val, int64_t n, const int32_t* __restrict__ gi,
                             const int32_t* __restrict__ gj, int32_t* __restrict__ pa, int32_t* __restrict__ pb) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k < n) { const uint32_t q = val[k]; pa[k] = gi[q]; pb[k] = gj[q]; }
}

__global__ void k_unit_count(const unsigned long long* __restrict__ ucnt, int64_t nbu, int64_t* __restrict__ nu) {
  const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (u < nbu) {
    const int64_t n = (int64_t)ucnt[u];
    nu[u] = n > 0 ? (n + UNIT_MAX - 1) / UNIT_MAX : 1;
  }
}

// multi[u] = 1 for the blocks that k_schur_finish completes: blocks split over several units, and every
// diagonal block (its damping and padding are applied there)
__global__ void k_unit_fill(const unsigned long long* __restrict__ ucnt, const int64_t* __restrict__ pstart,
                            const int64_t* __restrict__ ustart, int64_t nbu, const int32_t* __restrict__ up_row,
                            const int32_t* __restrict__ up_full, const int32_t* __restrict__ pcol,
                            int32_t* __restrict__ up_un, int32_t* __restrict__ un_se, int32_t* __restrict__ un_blk,
                            int64_t* __restrict__ multi) {
  const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (u > nbu) return;
  up_un[u] = (int32_t)ustart[u];
  if (u == nbu) return;
  const int64_t p0 = pstart[u], p1 = p0 + (int64_t)ucnt[u];
  for (int64_t w = ustart[u]; w < ustart[u + 1]; ++w) {
    const int64_t s = p0 + (w - ustart[u]) * UNIT_MAX;
    un_se[2 * w] = (int32_t)s;
    un_se[2 * w + 1] = (int32_t)(s + UNIT_MAX < p1 ? s + UNIT_MAX : p1);
    un_blk[w] = (int32_t)u;
  }
  multi[u] = (ustart[u + 1] - ustart[u] > 1 || pcol[up_full[u]] == up_row[u]) ? 1 : 0;
}

__global__ void k_multi_fill(const int64_t* __restrict__ flag, const int64_t* __restrict__ off, int64_t nbu,
                             int32_t* __restrict__ list) {
  const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (u < nbu && flag[u]) list[off[u]] = (int32_t)u;
}

// processing class of a unit (bits 30-31): 0 long (scheduled first), 1 other, 2 packable (a whole
// off-diagonal block of 1..PACK_MAX pairs, not a camera-plane block: its sums go straight to S).  Classes 0 and
// 1 run in the locality order of their block's row (bits 0-29, the row's rank), so that the units that read
// the slot records of the same features run close together in time and find them in L2; packable units keep
// block order (the packs take consecutive units).  The order changes no sum.
__global__ void k_unit_key(const int32_t* __restrict__ un_se, const int32_t* __restrict__ un_blk,
                           const int32_t* __restrict__ up_un, const int32_t* __restrict__ up_row,
                           const int32_t* __restrict__ up_full, const int32_t* __restrict__ pcol,
                           const int32_t* __restrict__ pair_b, const int32_t* __restrict__ rank, int64_t nun,
                           uint32_t* __restrict__ key, uint32_t* __restrict__ val) {
  const int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (w < nun) {
    const int n = un_se[2 * w + 1] - un_se[2 * w];
    const int u = un_blk[w];
    const bool diag = pcol[up_full[u]] == up_row[u];
    const bool single = up_un[u + 1] - up_un[u] == 1;
    // every pair of a packable unit carries no direct block (a block may mix pairs with and without one: the
    // camera-point block of a wireframe-coupled point has the lines' pairs and its own residuals' pair)
    bool nodirect = n >= 1 && n <= PACK_MAX;
    for (int k = 0; nodirect && k < n; ++k) nodirect = ((uint32_t)pair_b[un_se[2 * w] + k] >> PAIR_SHIFT) == 0u;
    const bool packable = !diag && single && nodirect;
    const uint32_t cls = n > UNIT_LONG ? 0u : (packable ? 2u : 1u);
    key[w] = (cls << 30) | (cls == 2u ? 0u : (uint32_t)rank[up_row[u]]);
    val[w] = (uint32_t)w;
  }
}

// validation and merge of one batch of residual records into the input-order arrays; a bad record leaves
// (merged index << 3 | code) in *err (atomicMin: the lowest index wins)
struct ObsGather {
  int kind, md;
  int64_t n, o;
  const int32_t *cam, *feat, *other;
  const double* meas;
  int64_t np, nl, nc, npl, nv, nsp, ncy, nco, nel, ncu;
  int8_t* kind_d;
  int32_t *cam_d, *feat_d, *grp_d;
  double* meas_d;
  unsigned long long* err;
};

__global__ void k_gather_obs(ObsGather a) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const int64_t j = a.o + i;
  const int k = a.kind;
  const bool is_point = (k == R_POINT || k == R_PLANE_POINT || k == R_P2L || k == R_PLANE_POINT3 ||
                         (k >= R_SPHERE_POINT && k <= R_CUB_POINT));
  int code = 0;
  const int32_t f = a.feat[i];
  if (f < 0 || f >= (is_point ? a.np : a.nl)) code = 1;
  int32_t c = -1;
  if (!code && res_has_cam(k)) {
    c = a.cam[i];
    if (c < 0 || c >= a.nc) code = 2;
  }
  int32_t g = -1;
  if (!code && (k == R_PLANE_POINT || k == R_PLANE_LINE || k == R_PLANE_POINT3 || k == R_PLANE_LINE3)) {
    g = a.other[i];
    if (g < 0 || g >= a.npl) code = 3;
  } else if (!code && k == R_VP) {
    g = a.other[i];
    if (g < 0 || g >= a.nv) code = 4;
  } else if (!code && ((k >= R_SPHERE_POINT && k <= R_CUB_POINT) || k == R_CUB_LINE)) {
    g = a.other[i];
    if (g < 0 || g >= (k == R_SPHERE_POINT ? a.nsp : k == R_CYL_POINT ? a.ncy : k == R_CONE_POINT ? a.nco
                       : k == R_ELL_POINT ? a.nel : a.ncu)) code = 7;
  } else if (!code && k == R_WF3D) {
    g = a.other[i];
    if (g < 0 || g >= a.np) code = 5;
  } else if (!code && (k == R_P2L || k == R_L2P) && a.other) {
    const int32_t q = a.other[i];
    if (q < 0 || q >= (k == R_P2L ? a.nl : a.np)) code = 5;
  }
  double m[4] = {0, 0, 0, 0};
  for (int t = 0; t < a.md; ++t) {
    m[t] = a.meas[(size_t)a.md * i + t];
    if (!code && !isfinite(m[t])) code = 6;
  }
  if (code) {
    atomicMin(a.err, ((unsigned long long)j << 3) | (unsigned long long)code);
    return;
  }
  a.kind_d[j] = (int8_t)k;
  a.feat_d[j] = is_point ? f : (int32_t)(a.np + f);
  a.cam_d[j] = c;
  a.grp_d[j] = g;
#pragma unroll
  for (int t = 0; t < 4; ++t) a.meas_d[4 * j + t] = m[t];
}

// per unit in processing order: (first pair, end pair, block position, unit id) and
// (mirror position << 2 | written directly << 1 | diagonal)
__global__ void k_unit_desc(const int32_t* __restrict__ order, const int32_t* __restrict__ un_se,
                            const int32_t* __restrict__ un_blk, const int32_t* __restrict__ up_un,
                            const int32_t* __restrict__ up_row, const int32_t* __restrict__ up_full,
                            const int32_t* __restrict__ up_mirror, const int32_t* __restrict__ pcol, int64_t nun,
                            int4* __restrict__ desc, int32_t* __restrict__ mflag) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= nun) return;
  const int w = order[g];
  const int u = un_blk[w];
  const int fpos = up_full[u];
  const bool diag = pcol[fpos] == up_row[u];
  const bool direct = !diag && up_un[u + 1] - up_un[u] == 1;
  desc[g] = make_int4(un_se[2 * w], un_se[2 * w + 1], fpos, w);
  mflag[g] = (up_mirror[u] << 2) | (direct ? 2 : 0) | (diag ? 1 : 0);
}

struct Permute {
  const uint32_t* order;
  const int8_t* kind;
  const int32_t *cam, *feat, *grp;
  const double4_32a* meas;
  int8_t* rkind;
  int32_t *rcam, *rfeat, *rgrp;
  double4_32a* rmeas;
  int64_t n;
};

__global__ void k_permute(Permute a) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= a.n) return;
  const uint32_t i = a.order[j];
  a.rkind[j] = a.kind[i];
  a.rcam[j] = a.cam[i];
  a.rfeat[j] = a.feat[i];
  a.rgrp[j] = a.grp[i];
  a.rmeas[j] = a.meas[i];
}

// The cost pass evaluates a point record together with the plane-induced record of the same point and camera
// (both project X into that camera): the first point record of each (feature, camera) run takes the run's
// first plane-induced record as its partner.  Records are feature-major and camera-sorted, so a run is
// contiguous.
__global__ void k_cost_partner(const int8_t* __restrict__ kind, const int32_t* __restrict__ cam,
                               const int32_t* __restrict__ feat, int64_t n, int32_t* __restrict__ partner,
                               uint8_t* __restrict__ attached, unsigned long long* __restrict__ nattached) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  partner[k] = -1;
  if (kind[k] != R_POINT) return;
  const int32_t f = feat[k], c = cam[k];
  int64_t b0 = k, b1 = k + 1;
  while (b0 > 0 && feat[b0 - 1] == f && cam[b0 - 1] == c) --b0;
  while (b1 < n && feat[b1] == f && cam[b1] == c) ++b1;
  for (int64_t j = b0; j < k; ++j)
    if (kind[j] == R_POINT) return;   // not the run's first point record
  for (int64_t j = b0; j < b1; ++j)
    if (kind[j] == R_PLANE_POINT) {
      partner[k] = (int32_t)j;
      attached[j] = 1;
      atomicAdd(nattached, 1ull);
      return;
    }
}

// cost order key: the kind, a point record with a partner before one without (the lanes of a warp then do the
// same work), attached plane-induced records last (the grid pass does not visit them)
__global__ void k_kind_key(const int8_t* __restrict__ kind, const int32_t* __restrict__ partner,
                           const uint8_t* __restrict__ attached, int64_t n, uint32_t* __restrict__ key,
                           uint32_t* __restrict__ val) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j < n) {
    key[j] = attached[j] ? 255u : 2u * (uint32_t)kind[j] + (partner[j] >= 0 ? 0u : 1u);
    val[j] = (uint32_t)j;
  }
}

__global__ void k_ent_type(int64_t na, int64_t nc, int64_t npl, int64_t nv, int64_t nsp, int64_t ncy, int64_t nco,
                           int64_t nel, int64_t ncu, int64_t nk, uint8_t* __restrict__ t) {
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= na) return;
  int64_t b = nc;
  uint8_t ty = ENT_CAM;
  if (a >= b) ty = ENT_PLANE;
  b += npl; if (a >= b) ty = ENT_VP;
  b += nv; if (a >= b) ty = ENT_SPHERE;
  b += nsp; if (a >= b) ty = ENT_CYL;
  b += ncy; if (a >= b) ty = ENT_CONE;
  b += nco; if (a >= b) ty = ENT_ELL1;
  b += nel; if (a >= b) ty = ENT_ELL2;
  b += nel; if (a >= b) ty = ENT_CUB1;
  b += ncu; if (a >= b) ty = ENT_CUB2;
  b += ncu; if (a >= b) ty = ENT_INTR;
  b += nk; if (a >= b) ty = ENT_JPT;
  t[a] = ty;
}

static ba_status read_i64(Problem& P, const int64_t* src, int64_t* dst) {
  CU(cudaMemcpyAsync(dst, src, sizeof(int64_t), cudaMemcpyDeviceToHost, P.stream));
  CU(cudaStreamSynchronize(P.stream));
  return BA_OK;
}

// A locality order of the block rows: reverse Cuthill-McKee over the camera-camera pattern of S (breadth-first
// from a camera of least degree, neighbours by ascending degree, every component in turn, reversed), the other
// rows after the cameras in index order.  Covisible cameras get nearby ranks.  rank[a] = position of row a.
static ba_status row_locality_rank(Problem& P, std::vector<int32_t>& rank) {
  const Dims& d = P.d;
  const int64_t na = d.na, nc = d.nc;
  rank.assign(na, 0);
  for (int64_t a = 0; a < na; ++a) rank[a] = (int32_t)a;
  if (nc < 3) return BA_OK;
  const int64_t ncol = P.h_prow_ptr[nc];
  std::vector<int32_t> col(ncol);
  CU(cudaMemcpyAsync(col.data(), P.col, sizeof(int32_t) * ncol, cudaMemcpyDeviceToHost, P.stream));
  CU(cudaStreamSynchronize(P.stream));
  std::vector<int32_t> deg(nc, 0);
  auto nbrs = [&](int64_t a, auto&& f) {
    for (int64_t q = P.h_prow_ptr[a]; q < P.h_prow_ptr[a + 1]; ++q) {
      const int32_t b = col[q];
      if (b < nc && b != a) f(b);
    }
  };
  for (int64_t a = 0; a < nc; ++a) nbrs(a, [&](int32_t) { ++deg[a]; });
  std::vector<int32_t> order;
  order.reserve(nc);
  std::vector<char> seen(nc, 0);
  std::vector<int32_t> byd(nc);
  std::iota(byd.begin(), byd.end(), 0);
  std::stable_sort(byd.begin(), byd.end(), [&](int32_t x, int32_t y) { return deg[x] < deg[y]; });
  std::vector<int32_t> next;
  for (int32_t st : byd) {
    if (seen[st]) continue;
    seen[st] = 1;
    size_t head = order.size();
    order.push_back(st);
    while (head < order.size()) {
      const int32_t a = order[head++];
      next.clear();
      nbrs(a, [&](int32_t b) { if (!seen[b]) { seen[b] = 1; next.push_back(b); } });
      std::stable_sort(next.begin(), next.end(), [&](int32_t x, int32_t y) { return deg[x] < deg[y]; });
      order.insert(order.end(), next.begin(), next.end());
    }
  }
  for (int64_t i = 0; i < nc; ++i) rank[order[nc - 1 - i]] = (int32_t)i;
  return BA_OK;
}

// ---------------------------------------------------------------------------
ba_status build_structure(Problem& P) {
  Dims& d = P.d;
  d.nc = (int64_t)P.h_cam.size() / 12;
  d.np = (int64_t)P.h_pts.size() / 3;
  d.nl = (int64_t)P.h_lin.size() / 6;
  d.npl = (int64_t)P.h_pln.size() / 4;
  d.nv = (int64_t)P.h_vps.size() / 3;
  d.nf = d.np + d.nl;
  // refined intrinsics (cam_dof 9): shared entities as set, else one per camera with the camera's values; every
  // camera's f, k1, k2 become a copy of its entity's
  if (P.opt.cam_dof == 9) {
    if (!P.intr_set) {
      P.h_intr.resize(3 * d.nc);
      P.h_cam_k.resize(d.nc);
      for (int64_t i = 0; i < d.nc; ++i) {
        for (int k = 0; k < 3; ++k) P.h_intr[3 * i + k] = P.h_cam[12 * i + 7 + k];
        P.h_cam_k[i] = (int32_t)i;
      }
    } else if ((int64_t)P.h_cam_k.size() != d.nc) {
      return fail(P, BA_ERR_ARG, "ba_set_intrinsics: intr_of_cam has " + std::to_string(P.h_cam_k.size()) +
                                     " entries for " + std::to_string(d.nc) + " cameras");
    }
    d.nk = (int64_t)P.h_intr.size() / 3;
    for (int64_t i = 0; i < d.nc; ++i)
      for (int k = 0; k < 3; ++k) P.h_cam[12 * i + 7 + k] = P.h_intr[3 * (size_t)P.h_cam_k[i] + k];
  }
  d.nsp = (int64_t)P.h_sph.size() / 4;
  d.ncy = (int64_t)P.h_cyl.size() / 7;
  d.nco = (int64_t)P.h_cone.size() / 7;
  d.nel = (int64_t)P.h_ell.size() / 10;
  d.ncu = (int64_t)P.h_cub.size() / 10;
  if ((d.ngs() || d.nbx()) && d.nk)
    return fail(P, BA_ERR_ARG, "refined intrinsics (cam_dof 9) together with spheres, cylinders, cones, ellipsoids "
                               "or cuboids are not supported");
  d.na = d.nc + d.npl + d.nv + d.ngs() + 2 * d.nbx() + d.nk;
  if (d.na > (int64_t)1 << 30 || d.nf > (int64_t)1 << 30) return fail(P, BA_ERR_ARG, "too many entities");
  // the pattern bitmap holds na x na bits
  int64_t wpr = (d.na + 31) / 32;
  if ((double)d.na * (double)wpr * 8.0 > 16e9)
    return fail(P, BA_ERR_ARG, "too many cameras and groups for the reduced-system pattern (" + std::to_string(d.na) + ")");

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

  // ---- spheres (c, r > 0), cylinders (Pluecker axis rescaled to |d| = 1, r > 0), cones (apex, unit axis, half-angle
  // in (0, pi/2)), SRF_STRIDE values each
  std::vector<double> srf(SRF_STRIDE * (size_t)d.ngs(), 0.0);
  for (int64_t i = 0; i < d.nsp; ++i) {
    const double* S_ = &P.h_sph[4 * i];
    if (!(S_[3] > 0) || !std::isfinite(S_[0] + S_[1] + S_[2] + S_[3]))
      return fail(P, BA_ERR_ARG, "sphere " + std::to_string(i) + ": the radius must be positive and finite");
    for (int k = 0; k < 4; ++k) srf[SRF_STRIDE * i + k] = S_[k];
  }
  for (int64_t i = 0; i < d.ncy; ++i) {
    const double* C_ = &P.h_cyl[7 * i];
    double* o = &srf[SRF_STRIDE * (d.nsp + i)];
    const double n = std::sqrt(C_[0] * C_[0] + C_[1] * C_[1] + C_[2] * C_[2]);
    if (!(n > 0) || !std::isfinite(n) || !(C_[6] > 0) || !std::isfinite(C_[6]))
      return fail(P, BA_ERR_ARG, "cylinder " + std::to_string(i) + ": zero axis direction or a radius that is not positive");
    for (int k = 0; k < 6; ++k) o[k] = C_[k] / n;
    const double dm = o[0] * o[3] + o[1] * o[4] + o[2] * o[5];   // keep m perpendicular to d
    for (int k = 0; k < 3; ++k) o[3 + k] -= dm * o[k];
    o[6] = C_[6];
  }
  for (int64_t i = 0; i < d.nco; ++i) {
    const double* K_ = &P.h_cone[7 * i];
    double* o = &srf[SRF_STRIDE * (d.nsp + d.ncy + i)];
    const double n = std::sqrt(K_[3] * K_[3] + K_[4] * K_[4] + K_[5] * K_[5]);
    if (!(n > 0) || !std::isfinite(n) || !(K_[6] > 0 && K_[6] < 1.5707963267948966))
      return fail(P, BA_ERR_ARG, "cone " + std::to_string(i) + ": zero axis or a half-angle outside (0, pi/2)");
    for (int k = 0; k < 3; ++k) { o[k] = K_[k]; o[3 + k] = K_[3 + k] / n; }
    o[6] = K_[6];
  }

  // ---- ellipsoids (q, c, s > 0) and cuboids (q, d_0..5): R row-major from the unit quaternion (w, x, y, z),
  // BOX_STRIDE values each
  std::vector<double> bx(BOX_STRIDE * (size_t)d.nbx(), 0.0);
  for (int64_t i = 0; i < d.nbx(); ++i) {
    const bool ell = i < d.nel;
    const double* G_ = ell ? &P.h_ell[10 * i] : &P.h_cub[10 * (i - d.nel)];
    double* o = &bx[BOX_STRIDE * i];
    const double qn = std::sqrt(G_[0] * G_[0] + G_[1] * G_[1] + G_[2] * G_[2] + G_[3] * G_[3]);
    bool bad = !(qn > 0) || !std::isfinite(qn);
    for (int k = 4; k < 10; ++k) bad |= !std::isfinite(G_[k]);
    if (ell) for (int k = 7; k < 10; ++k) bad |= !(G_[k] > 0);
    if (bad)
      return fail(P, BA_ERR_ARG, std::string(ell ? "ellipsoid " : "cuboid ") + std::to_string(ell ? i : i - d.nel) +
                                     (ell ? ": zero quaternion or a semi-axis that is not positive" : ": zero quaternion"));
    const double w = G_[0] / qn, x = G_[1] / qn, y = G_[2] / qn, z = G_[3] / qn;
    const double R[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                         2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                         2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)};
    for (int k = 0; k < 9; ++k) o[k] = R[k];
    for (int k = 0; k < 6; ++k) o[9 + k] = G_[4 + k];
  }

  // ---- residual records: validated and merged in input order on the device (below)
  int64_t nr = 0;
  for (auto& b : P.d_obs) nr += b.n;
  if (nr > (int64_t)INT32_MAX - 1) return fail(P, BA_ERR_ARG, "too many residuals");
  d.nr = nr;

  Scratch S(&P.alloc, P.stream);
  const int NT = 256;
  int64_t na = d.na, nf = d.nf;
  bool any_wf = false;
  for (auto& b : P.d_obs) any_wf |= b.kind == R_WF3D && b.n > 0;
  ba_status s;
  auto oom = [&]() { return fail(P, BA_ERR_OOM, "device allocation failed"); };

  // raw residual records (input order) on the device
  int8_t* kind_d = S.get<int8_t>(nr);
  int32_t *cam_d = S.get<int32_t>(nr), *feat_d = S.get<int32_t>(nr), *grp_d = S.get<int32_t>(nr);
  double* meas_d = S.get<double>(4 * nr);
  uint8_t* fixed_d = S.get<uint8_t>(d.nc);
  if (!kind_d || !cam_d || !feat_d || !grp_d || !meas_d || !fixed_d) return oom();
  {
    unsigned long long* err = S.get<unsigned long long>(1);
    if (!err) return oom();
    const unsigned long long none = ~0ull;
    CU(cudaMemcpyAsync(err, &none, sizeof(none), cudaMemcpyHostToDevice, P.stream));
    int64_t o = 0;
    for (auto& b : P.d_obs) {
      ObsGather g{b.kind, b.md, b.n, o, b.cam, b.feat, b.other, b.meas, d.np, d.nl, d.nc, d.npl, d.nv, d.nsp, d.ncy, d.nco, d.nel, d.ncu,
                  kind_d, cam_d, feat_d, grp_d, meas_d, err};
      k_gather_obs<<<grid_of(b.n, NT), NT, 0, P.stream>>>(g);
      o += b.n;
    }
    unsigned long long herr = none;
    CU(cudaMemcpyAsync(&herr, err, sizeof(herr), cudaMemcpyDeviceToHost, P.stream));
    CU(cudaStreamSynchronize(P.stream));
    if (herr != none) {
      // the lowest offending record of the merged input order names the error
      const int code = (int)(herr & 7ull);
      const int64_t j = (int64_t)(herr >> 3);
      int kk = 0;
      int64_t o2 = 0;
      for (auto& b : P.d_obs) {
        if (j < o2 + b.n) { kk = b.kind; break; }
        o2 += b.n;
      }
      const std::string ks = std::to_string(kk);
      if (code == 1) return fail(P, BA_ERR_ARG, "observation kind " + ks + ": feature id out of range");
      if (code == 2) return fail(P, BA_ERR_ARG, "observation kind " + ks + ": camera id out of range");
      if (code == 3) return fail(P, BA_ERR_ARG, "plane id out of range");
      if (code == 4) return fail(P, BA_ERR_ARG, "vp id out of range");
      if (code == 5) return fail(P, BA_ERR_ARG, "partner feature id out of range");
      if (code == 7) return fail(P, BA_ERR_ARG, "sphere, cylinder, cone, ellipsoid or cuboid id out of range");
      return fail(P, BA_ERR_ARG, "non-finite measurement");
    }
    P.release_obs();
  }
  if (d.nc) CU(cudaMemcpyAsync(fixed_d, P.h_fixed.data(), d.nc, cudaMemcpyHostToDevice, P.stream));

  // ---- points named by a 3D wireframe distance: entities of A after the intrinsics (ascending point id);
  // their residuals are keyed to a zero-dimension feature each, after the points and lines
  d.njp = 0;
  int32_t* fkey_d = feat_d;
  if (any_wf) {
    if (d.nk || d.ngs() || d.nbx())
      return fail(P, BA_ERR_ARG, "3D wireframe distances together with refined intrinsics or with spheres, cylinders, "
                                 "cones, ellipsoids or cuboids are not supported");
    int64_t *mark = S.get<int64_t>(d.np + 1), *rank = S.get<int64_t>(d.np + 1);
    fkey_d = S.get<int32_t>(nr);
    if (!mark || !rank || !fkey_d) return oom();
    CU(cudaMemsetAsync(mark, 0, sizeof(int64_t) * (d.np + 1), P.stream));
    k_mark_jpt<<<grid_of(nr, NT), NT, 0, P.stream>>>(kind_d, grp_d, nr, mark);
    if ((s = scan_excl(P, S, mark, rank, d.np))) return s;
    if ((s = read_i64(P, rank + d.np, &d.njp))) return s;
    P.jq = P.dnew<int32_t>(d.np);
    P.jp_pt = P.dnew<int32_t>(d.njp);
    if (!P.jq || !P.jp_pt) return oom();
    if (d.np) k_jq<<<grid_of(d.np, NT), NT, 0, P.stream>>>(mark, rank, d.np, P.jq, P.jp_pt);
    k_fkey<<<grid_of(nr, NT), NT, 0, P.stream>>>(feat_d, P.jq, d.np, d.nf, nr, fkey_d);
    d.na += d.njp;
    na = d.na;
    if (d.na > (int64_t)1 << 30) return fail(P, BA_ERR_ARG, "too many entities");
    wpr = (d.na + 31) / 32;
    if ((double)d.na * (double)wpr * 8.0 > 16e9)
      return fail(P, BA_ERR_ARG, "too many cameras, groups and wireframe-coupled points for the reduced-system "
                                 "pattern (" + std::to_string(d.na) + ")");
  }
  d.nfp = d.nf + d.njp;
  nf = d.nfp;

  // ---- feature-major order: stable sort by camera, then stable sort by feature
  uint32_t *key = S.get<uint32_t>(nr), *order = S.get<uint32_t>(nr), *k2 = S.get<uint32_t>(nr), *v2 = S.get<uint32_t>(nr);
  if (!key || !order || !k2 || !v2) return oom();
  if (nr) {
    k_iota_key<<<grid_of(nr, NT), NT, 0, P.stream>>>(cam_d, nr, 1, key, order);
    if ((s = radix_sort(P, S, key, order, k2, v2, nr, bits_for(d.nc + 1)))) return s;
    k_gather_key<<<grid_of(nr, NT), NT, 0, P.stream>>>(fkey_d, order, nr, key);
    if ((s = radix_sort(P, S, key, order, k2, v2, nr, bits_for(nf)))) return s;
  }
  // residual offsets per feature
  int64_t* cnt64 = S.get<int64_t>(std::max(nf, na) + 1);
  int64_t* off64 = S.get<int64_t>(std::max(nf, na) + 1);
  if (!cnt64 || !off64) return oom();
  CU(cudaMemsetAsync(cnt64, 0, sizeof(int64_t) * (nf + 1), P.stream));
  if (nr) k_count<<<grid_of(nr, NT), NT, 0, P.stream>>>(fkey_d, nr, (unsigned long long*)cnt64);
  if ((s = scan_excl(P, S, cnt64, off64, nf))) return s;
  P.fres_off = P.dnew<int32_t>(nf + 1);
  if (!P.fres_off) return oom();
  k_i64_to_i32<<<grid_of(nf + 1, NT), NT, 0, P.stream>>>(off64, nf + 1, P.fres_off);
  {
    int64_t v;
    if ((s = read_i64(P, off64 + d.np, &v))) return s;
    d.n_points_res_end = v;
  }

  // ---- slots
  int* err_d = S.get<int>(1);
  if (!err_d) return oom();
  CU(cudaMemsetAsync(err_d, 0, sizeof(int), P.stream));
  if (d.nk) {
    P.cam_k = P.dnew<int32_t>(d.nc);
    if (!P.cam_k) return oom();
    CU(cudaMemcpyAsync(P.cam_k, P.h_cam_k.data(), sizeof(int32_t) * d.nc, cudaMemcpyHostToDevice, P.stream));
  }
  const int64_t kbase = d.kbase();
  SlotArgs sa{(const int32_t*)order, P.fres_off, cam_d, grp_d, kind_d, fixed_d, nf, d.nc, d.npl, err_d, P.cam_k, kbase,
              d.sbase(), d.nsp, d.ncy, d.bbase(), d.nel, d.ncu, P.jq, d.jbase(), d.nf};
  int64_t* soff = S.get<int64_t>(nf + 1);
  if (!soff) return oom();
  k_slot_count<<<grid_of(nf, NT), NT, 0, P.stream>>>(sa, cnt64);
  if ((s = scan_excl(P, S, cnt64, soff, nf))) return s;
  int64_t ne;
  if ((s = read_i64(P, soff + nf, &ne))) return s;
  int herr = 0;
  CU(cudaMemcpyAsync(&herr, err_d, sizeof(int), cudaMemcpyDeviceToHost, P.stream));
  CU(cudaStreamSynchronize(P.stream));
  if (herr & 1)
    return fail(P, BA_ERR_ARG, "a feature may be associated with at most one plane, sphere, cylinder, cone, ellipsoid "
                               "or cuboid");
  if (herr & 2) return fail(P, BA_ERR_ARG, "a line may be associated with at most one VP");
  if (ne > (int64_t)INT32_MAX - 1) return fail(P, BA_ERR_ARG, "too many slots");
  d.ne = ne;
  P.fslot_off = P.dnew<int32_t>(nf + 1);
  P.slot_ent = P.dnew<int32_t>(ne); P.slot_feat = P.dnew<int32_t>(ne); P.slot_type = P.dnew<uint8_t>(ne);
  P.feat_plane_slot = P.dnew<int32_t>(nf);
  P.rslot_c = P.dnew<int32_t>(nr); P.rslot_g = P.dnew<int32_t>(nr);
  if (!P.fslot_off || !P.slot_ent || !P.slot_feat || !P.slot_type || !P.feat_plane_slot || !P.rslot_c || !P.rslot_g) return oom();
  if (d.nk || d.njp) {
    P.rslot_k = P.dnew<int32_t>(nr);
    if (!P.rslot_k) return oom();
  }
  SlotFill sf{P.fslot_off, P.slot_ent, P.slot_feat, P.feat_plane_slot, P.rslot_c, P.rslot_g, P.rslot_k, P.slot_type};
  k_slot_fill<<<grid_of(nf + 1, NT), NT, 0, P.stream>>>(sa, soff, sf);
  {
    int64_t v;
    if ((s = read_i64(P, soff + d.np, &v))) return s;
    P.line_slot0 = (int)v;
  }

  // ---- block pattern of S
  Bitmap bm{S.get<uint32_t>(na * wpr), wpr};
  int32_t* wpre = S.get<int32_t>(na * wpr);
  if (!bm.w || !wpre) return oom();
  CU(cudaMemsetAsync(bm.w, 0, sizeof(uint32_t) * na * wpr, P.stream));
  if ((s = build_relations(P))) return s;
  if (na) {
    k_pattern_diag<<<grid_of(na, NT), NT, 0, P.stream>>>(na, bm);
    if (nf) k_pattern_pairs<<<grid_of(nf, NT), NT, 0, P.stream>>>(P.fslot_off, P.slot_ent, nf, bm);
    if (P.nrel) k_pattern_rel<<<grid_of(P.nrel, NT), NT, 0, P.stream>>>(P.nrel, P.rel_ga, P.rel_gb, bm);
  }
  int64_t *full_cnt = S.get<int64_t>(na + 1), *pad_cnt = S.get<int64_t>(na + 1), *up_cnt = S.get<int64_t>(na + 1);
  int64_t *rowp = S.get<int64_t>(na + 1), *prow = S.get<int64_t>(na + 1), *uptr = S.get<int64_t>(na + 1);
  int32_t* nlow = S.get<int32_t>(na);
  if (!full_cnt || !pad_cnt || !up_cnt || !rowp || !prow || !uptr || !nlow) return oom();
  if (na) k_pattern_rows<<<grid_of(na, NT), NT, 0, P.stream>>>(na, bm, wpre, full_cnt, pad_cnt, up_cnt, nlow);
  if ((s = scan_excl(P, S, full_cnt, rowp, na))) return s;
  if ((s = scan_excl(P, S, pad_cnt, prow, na))) return s;
  if ((s = scan_excl(P, S, up_cnt, uptr, na))) return s;
  int64_t nbf, nbp, nbu;
  if ((s = read_i64(P, rowp + na, &nbf)) || (s = read_i64(P, prow + na, &nbp)) || (s = read_i64(P, uptr + na, &nbu))) return s;
  if (nbp > (int64_t)INT32_MAX - 1) return fail(P, BA_ERR_ARG, "too many blocks in the reduced system");
  d.nbf = nbf; d.nbp = nbp; d.nbu = nbu;
  P.row_ptr = P.dnew<int32_t>(na + 1); P.col = P.dnew<int32_t>(nbp); P.row_len = P.dnew<int32_t>(na);
  P.up_row = P.dnew<int32_t>(nbu); P.up_full = P.dnew<int32_t>(nbu); P.up_mirror = P.dnew<int32_t>(nbu);
  if (!P.row_ptr || !P.col || !P.row_len || !P.up_row || !P.up_full || !P.up_mirror) return oom();
  RowFill rf{prow, uptr, wpre, nlow, P.col, P.up_row, P.up_full, P.up_mirror, P.row_ptr, P.row_len, full_cnt};
  k_pattern_fill<<<grid_of(na + 1, NT), NT, 0, P.stream>>>(na, bm, rf);
  if ((s = relation_positions(P))) return s;
  P.h_prow_ptr.assign(na + 1, 0);
  P.h_row_len.assign(na, 0);
  CU(cudaMemcpyAsync(P.h_prow_ptr.data(), P.row_ptr, sizeof(int32_t) * (na + 1), cudaMemcpyDeviceToHost, P.stream));
  if (na) CU(cudaMemcpyAsync(P.h_row_len.data(), P.row_len, sizeof(int32_t) * na, cudaMemcpyDeviceToHost, P.stream));

  // ---- slot pairs per upper block, in feature order, cut into work items
  int64_t* poff = S.get<int64_t>(nf + 1);
  if (!poff) return oom();
  k_pair_count<<<grid_of(nf, NT), NT, 0, P.stream>>>(P.fslot_off, nf, cnt64);
  if ((s = scan_excl(P, S, cnt64, poff, nf))) return s;
  int64_t npair;
  if ((s = read_i64(P, poff + nf, &npair))) return s;
  if (npair > (int64_t)INT32_MAX - 1) return fail(P, BA_ERR_ARG, "too many Schur pairs");
  d.npair = npair;
  uint32_t *pkey = S.get<uint32_t>(npair), *pval = S.get<uint32_t>(npair);
  uint32_t *pk2 = S.get<uint32_t>(npair), *pv2 = S.get<uint32_t>(npair);
  int32_t *gi = S.get<int32_t>(npair), *gj = S.get<int32_t>(npair);
  unsigned long long* ucnt = S.get<unsigned long long>(nbu + 1);
  if (!pkey || !pval || !pk2 || !pv2 || !gi || !gj || !ucnt) return oom();
  CU(cudaMemsetAsync(ucnt, 0, sizeof(unsigned long long) * (nbu + 1), P.stream));
  PairGen pg{P.fslot_off, P.slot_ent, wpre, nlow, P.slot_type, P.cam_k, kbase, d.nf, poff, uptr, bm, nf, pkey, pval, gi, gj, ucnt};
  if (nf) k_pair_gen<<<grid_of(nf, NT), NT, 0, P.stream>>>(pg);
  if ((s = radix_sort(P, S, pkey, pval, pk2, pv2, npair, bits_for(nbu)))) return s;
  P.pair_a = P.dnew<int32_t>(npair); P.pair_b = P.dnew<int32_t>(npair);
  if (!P.pair_a || !P.pair_b) return oom();
  if (npair) k_pair_place<<<grid_of(npair, NT), NT, 0, P.stream>>>(pval, npair, gi, gj, P.pair_a, P.pair_b);
  int64_t* pstart = S.get<int64_t>(nbu + 1);
  if (!pstart) return oom();
  if ((s = scan_excl(P, S, (const int64_t*)ucnt, pstart, nbu))) return s;

  // ---- Schur work units: <= UNIT_MAX pairs of one block, long units first
  {
    int64_t *nuc = S.get<int64_t>(nbu + 1), *ustart = S.get<int64_t>(nbu + 1);
    int64_t *mflag = S.get<int64_t>(nbu + 1), *moff = S.get<int64_t>(nbu + 1);
    if (!nuc || !ustart || !mflag || !moff) return oom();
    if (nbu) k_unit_count<<<grid_of(nbu, NT), NT, 0, P.stream>>>(ucnt, nbu, nuc);
    if ((s = scan_excl(P, S, nuc, ustart, nbu))) return s;
    int64_t nun;
    if ((s = read_i64(P, ustart + nbu, &nun))) return s;
    d.nun = nun;
    P.up_un = P.dnew<int32_t>(nbu + 1); P.un_se = P.dnew<int32_t>(2 * nun); P.un_blk = P.dnew<int32_t>(nun);
    P.un_order = P.dnew<int32_t>(nun); P.upart = P.dnew<double>(48 * nun); P.unit_ctr = P.dnew<int>(1);
    if (!P.up_un || !P.un_se || !P.un_blk || !P.un_order || !P.upart || !P.unit_ctr) return oom();
    k_unit_fill<<<grid_of(nbu + 1, NT), NT, 0, P.stream>>>(ucnt, pstart, ustart, nbu, P.up_row, P.up_full, P.col,
                                                            P.up_un, P.un_se, P.un_blk, mflag);
    if ((s = scan_excl(P, S, mflag, moff, nbu))) return s;
    int64_t nmulti;
    if ((s = read_i64(P, moff + nbu, &nmulti))) return s;
    d.nmulti = nmulti;
    P.multi_blk = P.dnew<int32_t>(nmulti);
    if (!P.multi_blk) return oom();
    if (nbu) k_multi_fill<<<grid_of(nbu, NT), NT, 0, P.stream>>>(mflag, moff, nbu, P.multi_blk);
    uint32_t *uk = S.get<uint32_t>(nun), *uk2 = S.get<uint32_t>(nun), *uv2 = S.get<uint32_t>(nun);
    if (!uk || !uk2 || !uv2) return oom();
    if (nun) {
      std::vector<int32_t> hrank;
      if ((s = row_locality_rank(P, hrank))) return s;
      int32_t* rank_d = S.get<int32_t>(na);
      if (!rank_d) return oom();
      CU(cudaMemcpyAsync(rank_d, hrank.data(), sizeof(int32_t) * na, cudaMemcpyHostToDevice, P.stream));
      k_unit_key<<<grid_of(nun, NT), NT, 0, P.stream>>>(P.un_se, P.un_blk, P.up_un, P.up_row, P.up_full, P.col,
                                                       P.pair_b, rank_d, nun, uk, (uint32_t*)P.un_order);
      if ((s = radix_sort(P, S, uk, (uint32_t*)P.un_order, uk2, uv2, nun, 32))) return s;
    }
    if (nbp >= ((int64_t)1 << 29)) return fail(P, BA_ERR_ARG, "too many blocks in the reduced system");
    P.un_desc = P.dnew<int32_t>(4 * nun);
    P.un_mflag = P.dnew<int32_t>(nun);
    if (!P.un_desc || !P.un_mflag) return oom();
    if (nun)
      k_unit_desc<<<grid_of(nun, NT), NT, 0, P.stream>>>(P.un_order, P.un_se, P.un_blk, P.up_un, P.up_row, P.up_full,
                                                        P.up_mirror, P.col, nun, (int4*)P.un_desc, P.un_mflag);
    // packs: the packable units (the tail of the processing order, in block order) taken greedily while
    // their pairs stay contiguous and number at most PACK_MAX
    d.nun_main = nun;
    d.npack = 0;
    if (nun) {
      std::vector<uint32_t> hk(nun);
      CU(cudaMemcpyAsync(hk.data(), uk, sizeof(uint32_t) * nun, cudaMemcpyDeviceToHost, P.stream));
      CU(cudaStreamSynchronize(P.stream));
      const int64_t nmain = std::lower_bound(hk.begin(), hk.end(), 2u << 30) - hk.begin();
      const int64_t nsm = nun - nmain;
      if (nsm > 0) {
        std::vector<int32_t> hd(4 * nsm);
        CU(cudaMemcpyAsync(hd.data(), P.un_desc + 4 * nmain, sizeof(int32_t) * hd.size(), cudaMemcpyDeviceToHost,
                           P.stream));
        CU(cudaStreamSynchronize(P.stream));
        std::vector<int32_t> pk;
        for (int64_t i = 0; i < nsm;) {
          const int64_t i0 = i;
          const int32_t p0 = hd[4 * i];
          int32_t end = hd[4 * i + 1];
          for (++i; i < nsm && hd[4 * i] == end && hd[4 * i + 1] - p0 <= PACK_MAX; ++i) end = hd[4 * i + 1];
          pk.insert(pk.end(), {(int32_t)(nmain + i0), (int32_t)(i - i0), p0, end - p0});
        }
        P.pk_desc = P.dnew<int32_t>((int64_t)pk.size());
        if (!P.pk_desc) return oom();
        CU(cudaMemcpyAsync(P.pk_desc, pk.data(), sizeof(int32_t) * pk.size(), cudaMemcpyHostToDevice, P.stream));
        CU(cudaStreamSynchronize(P.stream));
        d.nun_main = nmain;
        d.npack = (int64_t)pk.size() / 4;
      }
    }
  }

  // ---- residual records in feature-major order
  P.rkind = P.dnew<int8_t>(nr); P.rcam = P.dnew<int32_t>(nr); P.rfeat = P.dnew<int32_t>(nr); P.rgrp = P.dnew<int32_t>(nr);
  P.meas64 = P.dnew<double>(4 * nr);
  if (!P.rkind || !P.rcam || !P.rfeat || !P.rgrp || !P.meas64) return oom();
  if (nr) {
    Permute pm{order, kind_d, cam_d, feat_d, grp_d, (const double4_32a*)meas_d, P.rkind, P.rcam, P.rfeat, P.rgrp,
               (double4_32a*)P.meas64, nr};
    k_permute<<<grid_of(nr, NT), NT, 0, P.stream>>>(pm);
  }
  // the cost pass visits the residuals kind by kind (feature-major inside a kind), so that the lanes of a
  // warp evaluate the same residual formula
  P.cost_order = P.dnew<int32_t>(nr);
  if (!P.cost_order) return oom();
  if (nr) {
    uint8_t* attached = S.get<uint8_t>(nr);
    unsigned long long* natt = S.get<unsigned long long>(1);
    P.cost_partner = P.dnew<int32_t>(nr);
    if (!attached || !natt || !P.cost_partner) return oom();
    CU(cudaMemsetAsync(attached, 0, nr, P.stream));
    CU(cudaMemsetAsync(natt, 0, sizeof(unsigned long long), P.stream));
    k_cost_partner<<<grid_of(nr, NT), NT, 0, P.stream>>>(P.rkind, P.rcam, P.rfeat, nr, P.cost_partner, attached, natt);
    k_kind_key<<<grid_of(nr, NT), NT, 0, P.stream>>>(P.rkind, P.cost_partner, attached, nr, key, (uint32_t*)P.cost_order);
    if ((s = radix_sort(P, S, key, (uint32_t*)P.cost_order, k2, v2, nr, 8))) return s;
    unsigned long long h = 0;
    CU(cudaMemcpyAsync(&h, natt, sizeof(h), cudaMemcpyDeviceToHost, P.stream));
    CU(cudaStreamSynchronize(P.stream));
    d.nr_cost = nr - (int64_t)h;
  } else {
    d.nr_cost = 0;
  }
  P.ent_type = P.dnew<uint8_t>(na);
  if (!P.ent_type) return oom();
  if (na) k_ent_type<<<grid_of(na, NT), NT, 0, P.stream>>>(na, d.nc, d.npl, d.nv, d.nsp, d.ncy, d.nco, d.nel, d.ncu,
                                                            d.nk, P.ent_type);

  // ---- parameters
#define UP(dst, src) if ((s = upload(P, dst, src)) != BA_OK) return s
  UP(P.cam_fixed, P.h_fixed);
  for (int k = 0; k < 2; ++k) {
    auto& S_ = P.ps[k];
    UP(S_.cam, P.h_cam); UP(S_.pts, P.h_pts); UP(S_.lin, P.h_lin); UP(S_.pln, P.h_pln); UP(S_.vps, P.h_vps);
    if (d.nk) UP(S_.intr, P.h_intr);
    if (d.ngs()) UP(S_.srf, srf);
    if (d.nbx()) UP(S_.bx, bx);
    S_.camD = P.dnew<double>(d.nc * CAM_STRIDE);
    S_.grpD = P.dnew<double>((d.npl + d.nv) * GRP_STRIDE);
    if (!S_.camD || !S_.grpD) return oom();
  }
  P.cur = 0;
#undef UP
  CU(cudaGetLastError());
  // the scratch buffers are released when this function returns: finish the work that reads them
  CU(cudaStreamSynchronize(P.stream));
  return BA_OK;
}

// ---------------------------------------------------------------------------
// typed storage of the reduced system (see TY_CC in ba_internal.cuh)
// per row: its camera, plane, VP and intrinsics columns (columns of a row are in entity order: cameras,
// planes, VPs, intrinsics entities)
__global__ void k_typed_count(int64_t na, int64_t nc, int64_t npl, int64_t kb, const int32_t* __restrict__ row_ptr,
                              const int32_t* __restrict__ row_len, const int32_t* __restrict__ col,
                              int32_t* __restrict__ cnt) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= na) return;
  int32_t n0 = 0, n1 = 0, n2 = 0, n3 = 0;
  for (int32_t q = row_ptr[r]; q < row_ptr[r] + row_len[r]; ++q) {
    const int32_t c = col[q];
    if (c < nc) ++n0; else if (c < nc + npl) ++n1; else if (c < kb) ++n2; else ++n3;
  }
  cnt[4 * r] = n0; cnt[4 * r + 1] = n1; cnt[4 * r + 2] = n2; cnt[4 * r + 3] = n3;
}

struct TypedFill {
  int64_t na, nc, npl, kb, gv;
  const int32_t *row_ptr, *prow_end, *row_len, *col, *cnt;
  const int32_t* rinfo;   // camera row: value and block offsets of its CC, CP, CV, CK runs (8); group row: GG block 0
  int64_t gg_val0;
  int32_t *sel, *tcol, *gg_col;
};

__global__ void k_typed_fill(TypedFill a) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= a.na) return;
  const int32_t q0 = a.row_ptr[r], len = a.row_len[r];
  const int32_t* ri = a.rinfo + 8 * r;
  const int32_t ncc = a.cnt[4 * r], ncp = a.cnt[4 * r + 1], ncv = a.cnt[4 * r + 2], nck = a.cnt[4 * r + 3];
  const int32_t nv = (int32_t)(a.kb - a.nc - a.npl);
  if (r < a.nc) {
    for (int32_t k = 0; k < len; ++k) {
      const int32_t c = a.col[q0 + k];
      if (c < a.nc) {
        a.sel[q0 + k] = ri[0] + 36 * k;
        a.tcol[ri[1] + k] = c;
      } else if (c < a.nc + a.npl) {
        const int32_t kk = k - ncc;
        a.sel[q0 + k] = ri[2] + 18 * kk;
        a.tcol[ri[3] + kk] = 3 * (c - (int32_t)a.nc);
      } else if (c < a.kb) {
        const int32_t kk = k - ncc - ncp;
        a.sel[q0 + k] = ri[4] + 12 * kk;
        a.tcol[ri[5] + kk] = 3 * (int32_t)a.npl + 2 * (c - (int32_t)(a.nc + a.npl));
      } else {
        const int32_t kk = k - ncc - ncp - ncv;
        a.sel[q0 + k] = ri[6] + 18 * kk;
        a.tcol[ri[7] + kk] = 3 * (int32_t)a.npl + 2 * nv + 3 * (c - (int32_t)a.kb);
      }
    }
    // padding blocks of the four runs (zero values): a camera-camera pad gathers the row's own u, a
    // camera-group pad points at the dummy group values
    for (int32_t k = ncc; k < (ncc + TCHUNK - 1) / TCHUNK * TCHUNK; ++k) a.tcol[ri[1] + k] = (int32_t)r;
    for (int32_t k = ncp; k < (ncp + TCHUNK - 1) / TCHUNK * TCHUNK; ++k) a.tcol[ri[3] + k] = (int32_t)a.gv;
    for (int32_t k = ncv; k < (ncv + TCHUNK - 1) / TCHUNK * TCHUNK; ++k) a.tcol[ri[5] + k] = (int32_t)a.gv;
    for (int32_t k = nck; k < (nck + TCHUNK - 1) / TCHUNK * TCHUNK; ++k) a.tcol[ri[7] + k] = (int32_t)a.gv;
  } else {
    const int32_t g0 = ri[0];
    for (int32_t k = 0; k < len; ++k) {
      const int32_t c = a.col[q0 + k];
      if (c >= a.nc) {
        const int32_t kk = k - ncc;
        a.sel[q0 + k] = (int32_t)(a.gg_val0 + 36 * (int64_t)(g0 + kk));
        a.gg_col[g0 + kk] = c;
      } else {
        // only the transpose is stored: camera row c's block of this group
        int32_t lo = a.row_ptr[c], hi = a.row_ptr[c] + a.row_len[c] - 1;
        while (lo < hi) {
          const int32_t mid = (lo + hi) >> 1;
          if (a.col[mid] < r) lo = mid + 1; else hi = mid;
        }
        const int32_t kc = lo - a.row_ptr[c];
        const int32_t* rc = a.rinfo + 8 * (int64_t)c;
        const int32_t cc = a.cnt[4 * (int64_t)c], cp = a.cnt[4 * (int64_t)c + 1], cv = a.cnt[4 * (int64_t)c + 2];
        const int32_t o = r < a.nc + a.npl ? rc[2] + 18 * (kc - cc)
                          : (r < a.kb ? rc[4] + 12 * (kc - cc - cp) : rc[6] + 18 * (kc - cc - cp - cv));
        a.sel[q0 + k] = (int32_t)((uint32_t)o | SEL_MIRROR);
      }
    }
  }
  for (int32_t q = q0 + len; q < a.prow_end[r]; ++q) a.sel[q] = -1;
}

SView sview_of(const Problem& P) {
  SView v;
  if (P.typed) {
    v.sel = P.sel;
    v.col = P.col;
    v.nc = P.d.nc;
    v.npl = P.d.npl;
    v.gg_val0 = P.gg_val0;
    v.kb = P.d.kbase();
  }
  return v;
}

ba_status build_typed_storage(Problem& P, TypedPlan& plan) {
  const Dims& d = P.d;
  const int64_t na = d.na, nc = d.nc;
  constexpr int NT = 128;
  auto oom = [&]() { return fail(P, BA_ERR_OOM, "device allocation failed"); };
  const int64_t kb = d.kbase();
  int32_t* cnt_d = P.dnew<int32_t>(4 * na);
  if (!cnt_d) return oom();
  k_typed_count<<<grid_of(na, NT), NT, 0, P.stream>>>(na, nc, d.npl, kb, P.row_ptr, P.row_len, P.col, cnt_d);
  std::vector<int32_t> cnt(4 * na);
  CU(cudaMemcpyAsync(cnt.data(), cnt_d, sizeof(int32_t) * cnt.size(), cudaMemcpyDeviceToHost, P.stream));
  CU(cudaStreamSynchronize(P.stream));
  // camera rows: four runs of whole chunks; group rows: their group-group blocks, unpadded
  std::vector<int32_t> rinfo(8 * na, 0);
  plan.row_chunk0.assign(nc + 1, 0);
  plan.chunks.clear();
  plan.chunk_w.clear();
  int64_t val = 0, blk = 0;
  const int wt[4] = {36, 40, 28, 40};   // products per block (and the scatter of a camera-group block)
  for (int64_t r = 0; r < nc; ++r) {
    for (int t = 0; t < 4; ++t) {
      const int64_t n = cnt[4 * r + t];
      const int64_t nch = (n + TCHUNK - 1) / TCHUNK;
      rinfo[8 * r + 2 * t] = (int32_t)val;
      rinfo[8 * r + 2 * t + 1] = (int32_t)blk;
      for (int64_t k = 0; k < nch; ++k) {
        plan.chunks.push_back(make_int4((int32_t)(val + k * TCHUNK * ty_vals(t)), (int32_t)(blk + k * TCHUNK), (int32_t)r, t));
        plan.chunk_w.push_back(wt[t] + (t == 0 && k == 0 ? 8 : 0));
      }
      val += nch * TCHUNK * ty_vals(t);
      blk += nch * TCHUNK;
      if (val > (int64_t)INT32_MAX / 2) return fail(P, BA_ERR_ARG, "reduced system too large for the typed storage");
    }
    plan.row_chunk0[r + 1] = (int32_t)plan.chunks.size();
  }
  const int64_t ng = na - nc;
  std::vector<int32_t> gg_ptr(ng + 1, 0);
  for (int64_t g = 0; g < ng; ++g) {
    const int64_t r = nc + g;
    rinfo[8 * r] = gg_ptr[g];
    gg_ptr[g + 1] = gg_ptr[g] + cnt[4 * r + 1] + cnt[4 * r + 2] + cnt[4 * r + 3];
  }
  P.gg_val0 = val;
  P.tvals = val + 36 * (int64_t)gg_ptr[ng];
  if (P.tvals > (int64_t)INT32_MAX / 2) return fail(P, BA_ERR_ARG, "reduced system too large for the typed storage");
  P.sel = P.dnew<int32_t>(d.nbp);
  P.tcol = P.dnew<int32_t>(std::max<int64_t>(blk, 1));
  P.gg_ptr = P.dnew<int32_t>(ng + 1);
  P.gg_col = P.dnew<int32_t>(std::max<int32_t>(gg_ptr[ng], 1));
  int32_t* rinfo_d = P.dnew<int32_t>(8 * na);
  int32_t* pend_d = P.dnew<int32_t>(na);
  if (!P.sel || !P.tcol || !P.gg_ptr || !P.gg_col || !rinfo_d || !pend_d) return oom();
  CU(cudaMemcpyAsync(rinfo_d, rinfo.data(), sizeof(int32_t) * rinfo.size(), cudaMemcpyHostToDevice, P.stream));
  CU(cudaMemcpyAsync(P.gg_ptr, gg_ptr.data(), sizeof(int32_t) * gg_ptr.size(), cudaMemcpyHostToDevice, P.stream));
  CU(cudaMemcpyAsync(pend_d, P.h_prow_ptr.data() + 1, sizeof(int32_t) * na, cudaMemcpyHostToDevice, P.stream));
  TypedFill f{na, nc, d.npl, kb, 3 * d.npl + 2 * d.nv + 3 * d.nk, P.row_ptr, pend_d, P.row_len, P.col, cnt_d, rinfo_d,
              P.gg_val0, P.sel, P.tcol, P.gg_col};
  k_typed_fill<<<grid_of(na, NT), NT, 0, P.stream>>>(f);
  CU(cudaGetLastError());
  CU(cudaStreamSynchronize(P.stream));
  return BA_OK;
}

}  // namespace ba
