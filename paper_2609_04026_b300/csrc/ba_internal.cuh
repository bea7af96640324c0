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
constexpr int SC = 20;  // camera slot: J_cam^T w J_plane (6 x 3, 18 values)
constexpr int SBS = 6;  // back-substitution record per slot (6 values, unpadded: padding cost more than it saved)

enum EntType : uint8_t { ENT_CAM = 0, ENT_PLANE = 1, ENT_VP = 2 };

constexpr int PCG_FLAG_TIMEOUT = 8;   // DevScalars::flags bit: a TMA copy of S did not complete in time

// scalars kept on the device so that PCG and the LM decision need no host round trip
struct DevScalars {
  double rz, rz_new, pAp, rr, bnorm2, alpha, beta, tol2;
  double E, Epx, Enew, Epxnew, pred, gTd, dHd;
  double lambda, nu, gain;
  int iters, max_iters, done, accepted;
  int flags;                 // bit 0: a landmark block needed extra damping; bit 1: non-finite value;
                             // bit 2: a block-Jacobi block fell back to its diagonal; bit 3: PCG copy timeout
  unsigned int counter[8];   // arrival counters of the last-block reductions
};

// the frozen problem structure (built once, K0) plus every device array
using Problem = ::ba_problem;

struct Dims {
  int64_t nc = 0, np = 0, nl = 0, npl = 0, nv = 0;
  int64_t nf = 0, na = 0, nr = 0, ne = 0, nbu = 0, nbf = 0, nbp = 0, npair = 0;  // nbf stored blocks, nbp padded
  int64_t nun = 0, nmulti = 0;   // Schur work units of the grid path; blocks split over several units
  int64_t nun_main = 0, npack = 0;   // units a warp takes alone (the rest are packed), and the packs
  int64_t n_points_res_end = 0;  // residuals of points are [0, this); lines follow
};

// kernel launchers (kernels.cu); T = double (FP64 path) or float (mixed path)
template <class T> void launch_prepare(Problem& P, bool candidate_only);
template <class T> void launch_linearize(Problem& P);
template <class T> void launch_invert(Problem& P, double lambda);
template <class T> void launch_schur(Problem& P, double lambda);
template <class T> void launch_precond(Problem& P);
template <class T> void launch_pcg(Problem& P);
template <class T> int pcg_blocks_per_sm(size_t smem);
template <class T> void pcg_allow_smem(size_t smem);
constexpr int PCG_CHUNK = 64;   // stored blocks per SpMV chunk (caller-layout path)

// position of entry e (row-major 6 x 6) of the block at padded position q in the storage of S: blocks are
// stored whole and in order, so a 32-block chunk is one contiguous run of 1152 values
__host__ __device__ __forceinline__ size_t s_idx(int64_t q, int e) { return (size_t)q * 36 + (size_t)e; }
template <class T> void launch_backsub(Problem& P);
void launch_candidate(Problem& P);
void launch_cost(Problem& P, bool candidate);
cudaError_t ensure_ln1p_table(cudaStream_t st);   // the FP64 cost's logarithm table on the current device
cudaError_t launch_ln1p_eval(cudaStream_t st, int64_t n, const double* x, double* y);
void launch_decide(Problem& P);

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
    double *camD = nullptr, *grpD = nullptr;   // rotation matrices / tangent bases (CAM_STRIDE / GRP_STRIDE)
  } ps[2];
  int cur = 0;
  // working-type (double or float) copies of the current parameters used by the linearisation
  void *camT = nullptr, *ptsT = nullptr, *linT = nullptr, *grpT = nullptr;
  uint8_t* cam_fixed = nullptr;
  // residuals, feature-major
  int8_t* rkind = nullptr;
  int32_t *rcam = nullptr, *rfeat = nullptr, *rgrp = nullptr, *rslot_c = nullptr, *rslot_g = nullptr;
  double* meas64 = nullptr;
  int32_t* cost_order = nullptr;   // residual indices sorted by kind (feature-major inside a kind)
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
  int32_t *pair_a = nullptr, *pair_b = nullptr;   // pair_b bit 31: camera-plane pair
  // grid-path Schur work units: pair range, block, processing order (long units first), first unit of
  // every block, and the blocks whose units leave FP64 partials (48 per unit in upart)
  int32_t *un_se = nullptr, *un_blk = nullptr, *un_order = nullptr, *up_un = nullptr, *multi_blk = nullptr;
  int32_t *un_desc = nullptr, *un_mflag = nullptr;   // per unit in processing order (4 ints; 1 int)
  // packs of small units (a whole off-diagonal block of at most PACK_MAX pairs each, not camera-plane):
  // the units [nun_main, nun) of the processing order, several to a warp; per pack int4
  // {first unit in processing order, units, first pair, pairs}, the pairs contiguous
  int32_t* pk_desc = nullptr;
  double* upart = nullptr;
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
  int pcg_grid = 0;
  size_t pcg_smem = 0;
  cudaError_t pcg_err = cudaSuccess;
  // numeric arrays
  void *slotW = nullptr, *slotH = nullptr, *slotG = nullptr, *slotC = nullptr, *slotZ = nullptr, *slotB = nullptr;
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
  int* win_state = nullptr;     // batched windows: device copy of (set, linearised, steps, accepted, converged)
  int batch_threads = 0, batch_grid = 0;  // launch shape of the last batched solve started from this problem
  double* red = nullptr;        // per-block partial sums of reductions
  int red_cap = 0;
  ba::DevScalars* S = nullptr;  // device scalars
  ba::DevScalars* hS = nullptr; // pinned host mirror

  cudaEvent_t ev[16] = {};
  int launches = 0;              // kernel launches since the start of the current step
};

namespace ba {
ba_status build_structure(Problem& P);   // structure.cu
// batched windows (kernels.cu, launched from batch.cu)
template <class T> void fill_window_desc(Problem& P, void* out);
template <class T> size_t window_desc_size();
template <class T> cudaError_t launch_windows(cudaStream_t st, const void* descs, const int* order, int nwin, int iters,
                                              int* queue, int threads, int grid, size_t smem);
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
