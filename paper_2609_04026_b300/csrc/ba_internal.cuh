// Internal declarations of libba: device buffers, the frozen problem structure,
// kernel launchers.  Host orchestration lives in api.cu, kernels in kernels.cu,
// the one-time structure build (the analogue of a sparse solver's symbolic
// analysis) in structure.cu.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/ba.h"
#include "residuals.cuh"

namespace ba {

// ---------------------------------------------------------------------------
// device memory: allocated through the caller's hooks (e.g. the framework's
// caching allocator) when given, else cudaMalloc; freed in the destructor
struct Alloc {
  void* (*fa)(size_t, void*) = nullptr;
  void (*ff)(void*, void*) = nullptr;
  void* ctx = nullptr;
  void* get(size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (fa) {
      // the kernels move records with 16-byte accesses and bulk copies: a hook's block must be aligned
      // like cudaMalloc's (256 bytes); a misaligned block is handed back and the allocation fails
      void* p = fa(bytes, ctx);
      if (p && ((uintptr_t)p & 255u)) {
        if (ff) ff(p, ctx);
        return nullptr;
      }
      return p;
    }
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    return p;
  }
  void put(void* p) {
    if (!p) return;
    if (ff) ff(p, ctx); else cudaFree(p);
  }
};

struct DBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

// block sizes of the padded reduced system: every entity of A occupies a 6-wide block
constexpr int BS = 6;
constexpr int BS2 = BS * BS;
// per-slot record strides (in elements of the slot type), padded to 16-byte multiples so that the
// linearisation writes whole records with 16-byte stores
constexpr int SW = 24;  // W^T (k x 6), k = 3 (point) or 4 (line)
// G and H share one 16-byte aligned record of SG values: J_a^T w r (6 values), then the upper triangle of
// the direct 6x6 block J_a^T w J_a (21 values) at offset HG_H, then one pad; H is addressed as a view at
// that offset with the same stride
constexpr int SG = 28;
constexpr int HG_H = 6;
constexpr int SH = SG;
constexpr int SB = 6;   // the whitened per-slot b part
constexpr int SC = 20;  // camera slot: J_cam^T w J_plane (6 x 3, 18 values); intrinsics slot: J_K^T w J_plane
                        // (3 x 3 in the first 9); with refined intrinsics a second camera record of this size
                        // holds J_cam^T w J_K (6 x 3) of the camera's own intrinsics entity
constexpr int SBS = 6;  // back-substitution record per slot (6 values, unpadded: padding cost more than it saved)
constexpr int SCS = 36; // camera slot of a feature on a sphere, cylinder or cone: J_cam^T w J_group (6 x 6, zero
                        // beyond the group's dimensions)

enum EntType : uint8_t {
  ENT_CAM = 0, ENT_PLANE = 1, ENT_VP = 2, ENT_INTR = 3, ENT_SPHERE = 4, ENT_CYL = 5, ENT_CONE = 6,
  ENT_ELL1 = 7, ENT_ELL2 = 8, ENT_CUB1 = 9, ENT_CUB2 = 10,  // a 9-parameter group's first (6) and second (3) entity
  ENT_JPT = 11   // a point that the 3D wireframe distance couples with a line feature (3)
};
// real dimensions of an entity block: camera pose 6, plane 3, VP 2, intrinsics (f, k1, k2) 3, sphere 4,
// cylinder 5, cone 6, a 9-parameter group's first entity 6 and second 3
__host__ __device__ __forceinline__ int ent_dims(int et) {
  return et == ENT_CAM ? 6 : et == ENT_VP ? 2 : et == ENT_SPHERE ? 4 : et == ENT_CYL ? 5
       : (et == ENT_CONE || et == ENT_ELL1 || et == ENT_CUB1) ? 6 : 3;
}
// a positional group that is not a plane (its camera couplings take the 6 x 6 CS records)
__host__ __device__ __forceinline__ bool ent_surface(int et) { return et >= ENT_SPHERE && et != ENT_ELL2 && et != ENT_CUB2; }
__host__ __device__ __forceinline__ bool ent_second(int et) { return et == ENT_ELL2 || et == ENT_CUB2; }
// direct coupling carried by a slot pair (pair_b bits 30-31): none, camera-plane (the camera slot's C record),
// camera-intrinsics (the camera slot's CK record, its own entity only), plane-intrinsics (the intrinsics slot's
// C record, transposed)
// camera-surface (the camera slot's CS record: a sphere, cylinder or cone of the feature)
// a 9-parameter group's two entities (the second entity's C record holds J_1^T w J_2, 6 x 3); PAIR_CK also
// carries a camera's block with a 9-parameter group's second entity (the camera slot's CK record; refined
// intrinsics are refused together with the other group types)
// The residuals of a point that the 3D wireframe distance makes an entity of A form a zero-dimension feature
// (zero Z records): its camera-point pairs carry PAIR_CK (the camera slot's CK record holds J_cam^T w J_point),
// its plane-point pair PAIR_PK (the point slot's C record holds J_point^T w J_plane)
constexpr uint32_t PAIR_CP = 1u, PAIR_CK = 2u, PAIR_PK = 3u, PAIR_CS = 4u, PAIR_G12 = 5u;
constexpr int PAIR_SHIFT = 29;
constexpr int32_t PAIR_SLOT = 0x1fffffff;

constexpr int PCG_FLAG_TIMEOUT = 8;   // DevScalars::flags bit: a bounded device-side wait of the PCG ran out

// Typed storage of the reduced system (the main path).  A camera row holds its camera-camera blocks (both
// triangles, 6 x 6), then its camera-plane blocks (6 x 3) and camera-VP blocks (6 x 2) at their real widths;
// each of the three runs is padded to whole chunks of 32 blocks.  The camera-group blocks are stored only
// there: a group row's camera part is the transpose, which the PCG forms from the camera rows (a scatter
// into per-warp accumulators of the group values).  A group row keeps its few group-group blocks (6 x 6).
constexpr int TY_CC = 0, TY_CP = 1, TY_CV = 2, TY_CK = 3;   // camera-intrinsics blocks: a fourth run (6 x 3)
constexpr int TCHUNK = 32;             // blocks per chunk (one per lane)
constexpr int GV_MAX = 1400;           // group values (3 per plane, 2 per VP, 3 per intrinsics entity) the typed
                                       // storage supports
constexpr int GV_PAD = 4;              // dummy group values behind the real ones (targets of padding blocks)
constexpr uint32_t SEL_MIRROR = 0x80000000u;   // sel[] flag: only the transposed copy of this block is stored
__host__ __device__ __forceinline__ int ty_vals(int ty) { return ty == TY_CC ? 36 : (ty == TY_CV ? 12 : 18); }

// Where the blocks of the reduced system live, addressed by their position q in the full padded block-CSR
// pattern (row_ptr / col).  Full storage (sel == null, batched windows): block q at 36 q, row-major 6 x 6.
// Typed storage: sel[q] as above; a stored block is 6 x 6 except a camera row's camera-group block, which is
// 6 x 3 (plane) or 6 x 2 (VP), row-major.
struct SView {
  const int32_t* sel = nullptr;
  const int32_t* col = nullptr;
  int64_t nc = 0, npl = 0, gg_val0 = 0;
  int64_t kb = 0;   // first intrinsics entity (nc + npl + nv)
};
// real width of a group entity's block: plane 3, VP 2, intrinsics 3
__host__ __device__ __forceinline__ int sview_gw(const SView& v, int64_t g) { return (g < v.nc + v.npl || g >= v.kb) ? 3 : 2; }
// width of the stored copy at typed offset o of a block in column c (the copy itself, not a mirror)
__host__ __device__ __forceinline__ int sview_width(const SView& v, int64_t o, int64_t c) {
  return (o < v.gg_val0 && c >= v.nc) ? sview_gw(v, c) : 6;
}
// the padded 6 x 6 block at position q of row r (zeros beyond a narrow block's width; the transpose of the
// stored copy when only the mirror is stored; all zeros for a padding position)
template <class T>
__host__ __device__ __forceinline__ void sview_load(const SView& v, const T* Sval, int64_t q, int64_t r, double (&out)[36]) {
  if (!v.sel) {
    for (int e = 0; e < 36; ++e) out[e] = (double)Sval[36 * q + e];
    return;
  }
  for (int e = 0; e < 36; ++e) out[e] = 0.0;
  const int32_t s = v.sel[q];
  if (s == -1) return;
  const int64_t o = (int64_t)(s & 0x7fffffff);
  if (!((uint32_t)s & SEL_MIRROR)) {
    const int w = sview_width(v, o, v.col[q]);
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < w; ++j) out[i * 6 + j] = (double)Sval[o + i * w + j];
  } else {
    const int w = sview_gw(v, r);   // the stored copy is camera row col[q]'s block of group r
    for (int i = 0; i < w; ++i)
      for (int j = 0; j < 6; ++j) out[i * 6 + j] = (double)Sval[o + j * w + i];
  }
}
// where a writer puts the block at position q: element offset and width, or width 0 when it is not stored there
struct BlkTarget {
  int64_t off;
  int w;
};
__host__ __device__ __forceinline__ BlkTarget sview_target(const SView& v, int64_t q) {
  if (!v.sel) return BlkTarget{36 * q, 6};
  const int32_t s = v.sel[q];
  if (s == -1 || ((uint32_t)s & SEL_MIRROR)) return BlkTarget{0, 0};
  return BlkTarget{(int64_t)s, sview_width(v, s, v.col[q])};
}

// scalars kept on the device so that PCG and the LM decision need no host round trip
struct DevScalars {
  double rz, rz_new, pAp, rr, bnorm2, alpha, beta, tol2;
  double E, Epx, Enew, Epxnew, pred, gTd, dHd;
  double lambda, nu, gain;
  int iters, max_iters, done, accepted;
  int flags;                 // bit 0: a landmark block needed extra damping; bit 1: non-finite value;
                             // bit 2: a block-Jacobi block fell back to its diagonal; bit 3: PCG wait timeout
  unsigned int counter[8];   // arrival counters of the last-block reductions
  unsigned int bar_count, bar_gen;   // grid barrier of the persistent PCG (count reset before every launch)
  unsigned long long bar_arrive;     // arrivals at the typed and stream PCGs' barriers in this launch (reset before it)
};

// the frozen problem structure (built once, K0) plus every device array
using Problem = ::ba_problem;

struct Dims {
  int64_t nc = 0, np = 0, nl = 0, npl = 0, nv = 0;
  int64_t nsp = 0, ncy = 0, nco = 0;   // spheres, cylinders, cones (A indices after the VPs, in that order)
  int64_t nel = 0, ncu = 0;            // ellipsoids, cuboids: two entities each (all first entities of a kind,
                                       // then its second ones), after the cones
  int64_t nk = 0;    // intrinsics entities (refined f, k1, k2; A indices after the groups)
  // the 3D wireframe distance: the points it names are entities of A (after the intrinsics); the residuals of
  // such a point form a zero-dimension feature of their own (one per point, after the points and lines)
  int64_t njp = 0;
  int64_t nfp = 0;   // features including those zero-dimension ones (nf: points and lines)
  int64_t jbase() const { return nc + npl + nv + nsp + ncy + nco + 2 * (nel + ncu) + nk; }
  int64_t ngs() const { return nsp + ncy + nco; }            // sphere, cylinder and cone groups
  int64_t nbx() const { return nel + ncu; }                  // 9-parameter groups
  int64_t sbase() const { return nc + npl + nv; }            // A index of the first sphere
  int64_t bbase() const { return sbase() + ngs(); }          // A index of the first ellipsoid's first entity
  int64_t kbase() const { return bbase() + 2 * nbx(); }      // A index of intrinsics entity 0
  int64_t nf = 0, na = 0, nr = 0, ne = 0, nbu = 0, nbf = 0, nbp = 0, npair = 0;  // nbf stored blocks, nbp padded
  int64_t nun = 0, nmulti = 0;   // Schur work units of the grid path; blocks split over several units
  int64_t nun_main = 0, npack = 0;   // units a warp takes alone (the rest are packed), and the packs
  int64_t n_points_res_end = 0;  // residuals of points are [0, this); lines follow
  int64_t nr_cost = 0;   // entries of the cost order the grid cost pass visits (a point's plane-induced record
                         // evaluated with its point record is not visited on its own)
};

// kernel launchers (kernels.cu); T = double (FP64 path) or float (mixed path)
template <class T> void launch_prepare(Problem& P, bool candidate_only, bool working_only = false);
template <class T> void launch_linearize(Problem& P);
template <class T> void launch_invert(Problem& P, double lambda);
template <class T> void launch_schur(Problem& P, double lambda);
template <class T> void launch_precond(Problem& P);
template <class T> void launch_pcg(Problem& P);
template <class T> int pcg_blocks_per_sm(size_t smem);
template <class T> void pcg_allow_smem(size_t smem);
template <class T> size_t pcg_typed_fixed_smem(int gv);
template <class T> size_t pcg_typed_gacc_bytes(int gv);
template <class T> int pcg_typed_blocks_per_sm(size_t smem);
constexpr int PCG_CHUNK = 64;   // stored blocks per SpMV chunk (caller-layout path)

// position of entry e (row-major 6 x 6) of the block at padded position q in the storage of S: blocks are
// stored whole and in order, so a 32-block chunk is one contiguous run of 1152 values
__host__ __device__ __forceinline__ size_t s_idx(int64_t q, int e) { return (size_t)q * 36 + (size_t)e; }
template <class T> void launch_backsub(Problem& P);
void launch_candidate(Problem& P);
void launch_cost(Problem& P, bool candidate);
cudaError_t ensure_ln1p_table(cudaStream_t st);   // the FP64 cost's logarithm table on the current device
cudaError_t launch_ln1p_eval(cudaStream_t st, int64_t n, const double* x, double* y);
cudaError_t fma_probe(int precision, double* tflops, cudaStream_t st);   // FP32 / FP64 FMA throughput
void launch_decide(Problem& P);
cudaError_t launch_convert(cudaStream_t st, int64_t n, const double* a, float* b);   // b = (float)a

}  // namespace ba

// The problem object (opaque to the ABI).
struct ba_problem {
  ba_options opt;
  std::string err;
  ba::Alloc alloc;
  cudaStream_t stream = nullptr;
  int device = 0;
  bool frozen = false;
  bool have_lin = false;     // linearisation valid for the current parameters
  bool have_reduced = false;
  double last_lambda = 0;

  // host staging of inputs until the structure is frozen
  std::vector<double> h_cam;      // n x 12: q(4) t(3) f k1 k2 ppx ppy
  std::vector<uint8_t> h_fixed;
  std::vector<double> h_pts, h_lin, h_pln, h_vps;
  std::vector<double> h_sph, h_cyl, h_cone;   // spheres (4), cylinders (7), cones (7) as added
  std::vector<double> h_ell, h_cub;           // ellipsoids (q, c, s), cuboids (q, d_0..5): 10 each as added
  std::vector<int32_t> h_rel;     // inter-group relations as added: 5 per relation (kind_a, a, kind_b, b, type)
  // shared intrinsics (ba_set_intrinsics): entity values (3 each) and every camera's entity
  std::vector<double> h_intr;
  std::vector<int32_t> h_cam_k;
  bool intr_set = false;
  // residual records as added, copied to the device at add time (validated and merged by the structure build,
  // which releases them); cam is null for VP records, other may be null, meas holds n x meas_dim values
  struct ObsBatch {
    int kind = 0, md = 0;
    int64_t n = 0;
    int32_t *cam = nullptr, *feat = nullptr, *other = nullptr;
    double* meas = nullptr;
  };
  std::vector<ObsBatch> d_obs;
  void release_obs() {
    for (auto& b : d_obs) { alloc.put(b.cam); alloc.put(b.feat); alloc.put(b.other); alloc.put(b.meas); }
    d_obs.clear();
  }

  ba::Dims d;
  std::vector<ba::DBuf> bufs;
  void* dalloc(size_t bytes);
  template <class X> X* dnew(int64_t n) { return (X*)dalloc(sizeof(X) * (size_t)(n > 0 ? n : 1)); }

  // ---- device arrays
  // parameters: two FP64 sets (current / candidate), each with its FP64 derived per-entity data
  struct ParamSet {
    double *cam = nullptr, *pts = nullptr, *lin = nullptr, *pln = nullptr, *vps = nullptr;
    double* intr = nullptr;   // intrinsics entities (f, k1, k2), refined intrinsics only; each camera's f, k1, k2
                              // in cam is a copy of its entity's values
    double* srf = nullptr;    // surface groups, SRF_STRIDE values each: sphere (c, r), cylinder (d, m, r), cone
                              // (apex, axis, half-angle)
    double* bx = nullptr;     // ellipsoids then cuboids, BOX_STRIDE values each: R row-major, then (c, s) or d_0..5
    double *camD = nullptr, *grpD = nullptr;   // rotation matrices / tangent bases (CAM_STRIDE / GRP_STRIDE)
  } ps[2];
  int cur = 0;
  // working-type (double or float) copies of the current parameters used by the linearisation
  void *camT = nullptr, *ptsT = nullptr, *linT = nullptr, *grpT = nullptr, *srfT = nullptr, *bxT = nullptr;
  uint8_t* cam_fixed = nullptr;
  int32_t* cam_k = nullptr;   // per camera its intrinsics entity (refined intrinsics only)
  int32_t* jq = nullptr;      // per point its index among the wireframe-coupled points, or -1
  int32_t* jp_pt = nullptr;   // per wireframe-coupled point its point id
  // residuals, feature-major
  int8_t* rkind = nullptr;
  int32_t *rcam = nullptr, *rfeat = nullptr, *rgrp = nullptr, *rslot_c = nullptr, *rslot_g = nullptr;
  int32_t* rslot_k = nullptr;   // per residual the slot of its camera's intrinsics entity (or -1)
  double* meas64 = nullptr;
  int32_t* cost_order = nullptr;   // residual indices sorted by kind (feature-major inside a kind)
  int32_t* cost_partner = nullptr; // per point record, the plane-induced record of the same point and camera
                                   // that the cost pass evaluates with it (pi(C, X) once), or -1
  void* measT = nullptr;
  int32_t *fres_off = nullptr, *fslot_off = nullptr;
  int32_t *slot_ent = nullptr, *slot_feat = nullptr;
  uint8_t* slot_type = nullptr;
  int32_t* feat_plane_slot = nullptr;
  uint8_t* ent_type = nullptr;
  // reduced system pattern: padded, interleaved storage (row_ptr / col over padded positions)
  int32_t *row_ptr = nullptr, *col = nullptr;
  std::vector<int32_t> h_prow_ptr, h_row_len;
  int32_t *up_row = nullptr, *up_full = nullptr, *up_mirror = nullptr;
  int32_t *pair_a = nullptr, *pair_b = nullptr;   // pair_b bits 30-31: the pair's direct coupling (PAIR_CP ...)
  // grid-path Schur work units: pair range, block, processing order (long units first), first unit of
  // every block, and the blocks whose units leave FP64 partials (48 per unit in upart)
  int32_t *un_se = nullptr, *un_blk = nullptr, *un_order = nullptr, *up_un = nullptr, *multi_blk = nullptr;
  int32_t *un_desc = nullptr, *un_mflag = nullptr;   // per unit in processing order (4 ints; 1 int)
  // packs of small units (a whole off-diagonal block of at most PACK_MAX pairs each, not camera-plane):
  // the units [nun_main, nun) of the processing order, several to a warp; per pack int4
  // {first unit in processing order, units, first pair, pairs}, the pairs contiguous
  int32_t* pk_desc = nullptr;
  double* upart = nullptr;
  int* unit_ctr = nullptr;   // the Schur unit kernel's work counter (reset before each launch)
  int line_slot0 = 0;           // first slot of a line feature
  // persistent PCG partition: CTA c owns block rows [cta_row0[c], cta_row0[c+1]); row r's stored blocks are
  // cut into chunks [chunk_beg[q], chunk_beg[q+1]) for q in [row_chunk0[r], row_chunk0[r+1])
  int32_t *cta_row0 = nullptr, *row_chunk0 = nullptr, *chunk_beg = nullptr;
  // streaming PCG partition: CTA c multiplies chunks [q0, q1) touching block rows [t0, t1), stored as
  // int4 {q0, q1, t0, t1}; a row cut by a CTA boundary belongs to the CTA holding its first chunk, and
  // the other CTAs leave their partial sums of it in pcg_carry (6 doubles per CTA)
  int32_t* cta_part = nullptr;
  double* pcg_carry = nullptr;
  float pcg_keep_frac = 0.f;   // fraction of S the PCG keeps resident in L2 across iterations
  // typed storage (see TY_CC): sel[q] = element offset of the stored copy of the block at full padded position q
  // (| SEL_MIRROR when only its transpose is stored, -1 for padding); per typed block its column code (camera
  // entity, or the group value offset of a camera-group block); per chunk {value offset, first block, row,
  // type}; per group row its group-group blocks; per CTA its slice of group rows; the group-value table
  bool typed = false;
  int gv = 0;                    // group values 3 npl + 2 nv
  int32_t *sel = nullptr, *tcol = nullptr, *gg_ptr = nullptr, *gg_col = nullptr, *cta_gs = nullptr, *gv_idx = nullptr;
  int4* tchunk = nullptr;
  int64_t tvals = 0, gg_val0 = 0;   // values of the typed storage; first value of the group-group region
  double* part_g = nullptr;      // per group value, every CTA's share of the scatter (gv x G)
  // inter-group relations: per relation its two group entities (A indices) and type; per group entity the
  // relations it takes part in (relation << 1 | side, in relation order); the distinct pairs of entities with
  // their relations and the full positions of both blocks; linearisation (double): r (3), J_a, J_b (3 x 6
  // each, padded), IRLS weight; per group entity the summed J^T w J (36) and J^T w r (6)
  int64_t nrel = 0, nrelpair = 0;
  int32_t *rel_ga = nullptr, *rel_gb = nullptr, *rel_type = nullptr, *grel_ptr = nullptr, *grel_idx = nullptr;
  int32_t *rp_ptr = nullptr, *rp_idx = nullptr, *rp_pos = nullptr;
  double *rel_lin = nullptr, *relH = nullptr, *relG = nullptr;
  int pcg_grid = 0;
  int pcg_nown = 0;              // typed PCG: the most values any CTA owns (its shared-memory vector room)
  size_t pcg_smem = 0;
  cudaError_t pcg_err = cudaSuccess;
  // numeric arrays
  void *slotW = nullptr, *slotH = nullptr, *slotG = nullptr, *slotC = nullptr, *slotZ = nullptr, *slotB = nullptr;
  void* slotCK = nullptr;       // refined intrinsics: per camera slot J_cam^T w J_K of its own entity (SC)
  void* slotCS = nullptr;       // surface groups: per camera slot J_cam^T w J_group of the feature's surface (SCS)
  void* slotBS = nullptr;       // back-substitution: per slot W da (4), G.da, da^T H da + 2 da^T C dplane
  double *featV = nullptr, *featg = nullptr, *featVinv = nullptr, *featu = nullptr, *featL = nullptr, *dfeat = nullptr;
  void *Sval = nullptr, *Minv = nullptr;
  double *bvec = nullptr, *Dg = nullptr, *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *Ap = nullptr;
  double* svec = nullptr;       // PCG: s = S p (Chronopoulos-Gear form)
  float2* phl = nullptr;        // mixed path: p split into (hi, lo) floats for the SpMV
  int32_t* row_len = nullptr;   // stored (non-padding) blocks per row of S
  double* sdiag = nullptr;      // diagonal of S (after damping), 6 per entity
  // learned correction of the block-Jacobi preconditioner
  float* pre_params = nullptr;  // network parameters (float)
  void *pre_w1 = nullptr, *pre_w2 = nullptr;  // weights as bf16 for inference
  float* pre_X = nullptr;       // features, 32 per block row
  uint8_t* pre_mask = nullptr;  // real dimensions per block row
  int* pre_fallbacks = nullptr; // blocks that fell back to block-Jacobi in the last build
  bool pre_ready = false;
  int* win_state = nullptr;     // batched windows: device copy of (set, linearised, steps, accepted, converged,
                                // pad, then the window's device time in ns as a 64-bit value at int 6)
  uint64_t serial = 0;          // unique per problem (a batch is identified by its windows' serials)
  // the last batch started from this problem: its instantiated graph and the buffers the graph's kernel reads,
  // kept so that the same batch launched again reuses them
  struct BatchGraph {
    std::vector<uint64_t> key;
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    cudaStream_t stream = nullptr;
    void *desc = nullptr, *order = nullptr, *queue = nullptr;
    int threads = 0, grid = 0, nct = 0, nbig = 0;
  } bgraph;
  int batch_threads = 0, batch_grid = 0;  // launch shape of the last batched solve started from this problem
  int batch_nct = 1, batch_nbig = 0;      // and its CTAs per window, windows run on clusters
  double* red = nullptr;        // per-block partial sums of reductions
  int red_cap = 0;
  ba::DevScalars* S = nullptr;  // device scalars
  ba::DevScalars* hS = nullptr; // pinned host mirror

  cudaEvent_t ev[16] = {};
  // the candidate's linearisation, made on a second stream beside the FP64 cost pass of the step that forms the
  // candidate; valid for the next step when the candidate is accepted
  cudaStream_t side = nullptr;
  cudaEvent_t sev[4] = {};   // fork, side start, side end (timing), join
  bool spec_lin = false;      // the last step linearised its candidate
  float spec_ms = 0.f;        // device time of that linearisation (on the side stream, overlapping the cost)
  int launches = 0;              // kernel launches since the start of the current step
};

namespace ba {
ba_status build_structure(Problem& P);   // structure.cu
// inter-group relations (relations.cu): device lists at freeze, linearisation, their share of S, b, the cost
// and the predicted decrease
ba_status build_relations(Problem& P);
ba_status relation_positions(Problem& P);
void launch_rel_linearize(Problem& P);
template <class T> void launch_rel_offdiag(Problem& P);
void launch_rel_cost(Problem& P, bool candidate);
void launch_rel_pred(Problem& P);
// typed storage of the reduced system (structure.cu): per full position its stored copy, column codes of the
// typed blocks, and the host plan of chunks; see TY_CC
struct TypedPlan {
  std::vector<int32_t> row_chunk0;   // camera row r's chunks [row_chunk0[r], row_chunk0[r + 1])
  std::vector<int32_t> chunk_w;      // per chunk its arithmetic weight (for the CTA partition)
  std::vector<int4> chunks;          // per chunk {value offset, first block, camera row, type}
};
ba_status build_typed_storage(Problem& P, TypedPlan& plan);
SView sview_of(const Problem& P);
// batched windows (kernels.cu, launched from batch.cu)
template <class T> void fill_window_desc(Problem& P, void* out);
template <class T> size_t window_desc_size();
template <class T> cudaError_t launch_windows(cudaStream_t st, const void* descs, const int* order, int nwin, int nbig,
                                              int iters, int* queue, int threads, int grid, size_t smem, int nct);
template <class T> int window_clusters(int threads, size_t smem, int nct);
template <class T> int windows_per_sm(int threads, size_t smem);
// learned preconditioner (precond.cu)
ba_status precond_set_weights(Problem& P, const float* host_params);
ba_status precond_alloc_features(Problem& P);
template <class T> void launch_pre_features(Problem& P);
template <class T> void launch_pre_learned(Problem& P);

// raw-pointer launchers (kernels.cu) for the allocation-free PCG entry point (noalloc.cu)
cudaError_t launch_precond_raw_f64(cudaStream_t st, int64_t na, const int32_t* row_ptr, const int32_t* col,
                                   const double* Sval, double* Minv, DevScalars* S);
int pcg_occupancy_f64(size_t smem);
cudaError_t launch_pcg_raw_f64(cudaStream_t st, int grid, size_t smem, int64_t na, const int32_t* col,
                               const int32_t* cta_row0, const int32_t* row_chunk0, const int32_t* chunk_beg,
                               const double* Sval, const double* Minv, const double* b, double* x, double* r,
                               double* z, double* p, double* Ap, double* part, DevScalars* S, double tol,
                               int max_iters);
}
