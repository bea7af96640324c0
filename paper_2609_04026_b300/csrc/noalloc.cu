// Allocation-free block-Jacobi PCG on a caller-supplied reduced system.
//
// Some callers cannot allocate device memory while they run: a solver embedded in
// a process whose memory is handed out once by its own arena (a real-time mapping
// or robotics stack with a fixed budget), or code that must not call cudaMalloc
// from inside its own per-frame loop.  This entry point runs the same persistent
// PCG kernel as the rest of the library, but every scratch vector lives in one
// file-scope device array of fixed size, so a call performs no cudaMalloc /
// cudaFree and no allocating library call.
//
// The array is global state: every GPU that loads the library holds it until the
// process exits, every call shares it (a call keeps the previous call's contents
// and sets what it needs before use), and calls whose GPU work overlaps race on it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "ba_internal.cuh"

using namespace ba;

namespace {

constexpr int64_t kMaxRows = 4096;                  // block rows (6 wide) of S
constexpr int64_t kMaxBlocks = int64_t(1) << 22;    // stored 6x6 blocks of S
constexpr int64_t kMaxChunks = kMaxBlocks / PCG_CHUNK + kMaxRows;
constexpr int kMaxGrid = 1024;
constexpr int kMaxDevices = 64;

struct Scratch {
  double r[6 * kMaxRows], z[6 * kMaxRows], p[6 * kMaxRows], Ap[6 * kMaxRows];
  double Minv[36 * kMaxRows];
  double part[6 * kMaxGrid];
  int32_t row_ptr[kMaxRows + 1];
  int32_t cta_row0[kMaxGrid + 1];
  int32_t row_chunk0[kMaxRows + 1];
  int32_t chunk_beg[kMaxChunks + 1];
  DevScalars S;
};

// the scratch array (about 2.3 MB per GPU)
static __device__ __align__(256) unsigned char g_pcg_scratch[sizeof(Scratch)];

// host copies of the partition, filled under the lock, then copied into the scratch array
struct HostPlan {
  int32_t cta_row0[kMaxGrid + 1];
  int32_t row_chunk0[kMaxRows + 1];
  int32_t chunk_beg[kMaxChunks + 1];
};
static HostPlan g_plan;
static std::mutex g_lock;
static void* g_dev_scratch[kMaxDevices];   // device address of g_pcg_scratch, per device

// every row has its diagonal block and every column index is in range -> flags stay 0
__global__ void k_check_pattern(int64_t n, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ cols,
                                DevScalars* S) {
  int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= n) return;
  bool diag = false;
  for (int q = row_ptr[a]; q < row_ptr[a + 1]; ++q) {
    const int c = cols[q];
    if (c < 0 || c >= n) { atomicOr(&S->flags, 16); return; }
    diag |= (c == a);
  }
  if (!diag) atomicOr(&S->flags, 32);
}

int set_msg(char* err, size_t len, const char* m) {
  if (err && len) {
    std::snprintf(err, len, "%s", m);
  }
  return 0;
}

}  // namespace

extern "C" ba_status ba_pcg_solve_static(int64_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* cols,
                                         const double* vals, const double* b, double* x, double rel_tol,
                                         int max_iters, void* cuda_stream, int* iters, double* rel, char* err,
                                         size_t err_len) {
  if (n <= 0 || n > kMaxRows) {
    set_msg(err, err_len, "ba_pcg_solve_static: n_block_rows must be in [1, 4096]");
    return BA_ERR_ARG;
  }
  if (nnz < n || nnz > kMaxBlocks) {
    set_msg(err, err_len, "ba_pcg_solve_static: nnz_blocks must be in [n_block_rows, 4194304]");
    return BA_ERR_ARG;
  }
  if (!row_ptr || !cols || !vals || !b || !x || !(rel_tol > 0) || max_iters <= 0) {
    set_msg(err, err_len, "ba_pcg_solve_static: null array, rel_tol <= 0 or max_iters <= 0");
    return BA_ERR_ARG;
  }
  if (row_ptr[0] != 0 || row_ptr[n] != nnz) {
    set_msg(err, err_len, "ba_pcg_solve_static: row_ptr must start at 0 and end at nnz_blocks");
    return BA_ERR_ARG;
  }
  for (int64_t r = 0; r < n; ++r)
    if (row_ptr[r + 1] <= row_ptr[r]) {
      set_msg(err, err_len, "ba_pcg_solve_static: every block row needs at least its diagonal block");
      return BA_ERR_ARG;
    }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  std::lock_guard<std::mutex> guard(g_lock);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    set_msg(err, err_len, "ba_pcg_solve_static: no usable CUDA device");
    return BA_ERR_CUDA;
  }
  // set-up, once per device, with that device current: the device address of the scratch array
  if (!g_dev_scratch[dev]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_pcg_scratch);
    if (e != cudaSuccess || !ptr) {
      cudaGetLastError();
      set_msg(err, err_len, "ba_pcg_solve_static: cudaGetSymbolAddress failed");
      return BA_ERR_CUDA;
    }
    g_dev_scratch[dev] = ptr;
  }
  Scratch* W = (Scratch*)g_dev_scratch[dev];

  // partition of the block rows over the CTAs of the persistent kernel (balanced by stored blocks)
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    set_msg(err, err_len, "ba_pcg_solve_static: device query failed");
    return BA_ERR_CUDA;
  }
  int64_t nch = 0;
  g_plan.row_chunk0[0] = 0;
  for (int64_t r = 0; r < n; ++r) {
    const int32_t len = row_ptr[r + 1] - row_ptr[r];
    const int32_t k = std::max<int32_t>(1, (len + PCG_CHUNK - 1) / PCG_CHUNK);
    for (int32_t j = 0; j < k; ++j) g_plan.chunk_beg[nch + j] = row_ptr[r] + j * PCG_CHUNK;
    nch += k;
    g_plan.row_chunk0[r + 1] = (int32_t)nch;
  }
  g_plan.chunk_beg[nch] = (int32_t)nnz;
  int per_sm = std::max(1, std::min(2, pcg_occupancy_f64(48 * 1024)));
  int64_t G = std::max<int64_t>(1, std::min<int64_t>({(int64_t)sms * per_sm, n, (int64_t)kMaxGrid}));
  size_t smem = 0;
  for (;;) {
    double total = 0, acc = 0;
    for (int64_t r = 0; r < n; ++r) total += (row_ptr[r + 1] - row_ptr[r]) + 2.0;
    int64_t m = 1;
    g_plan.cta_row0[0] = 0;
    for (int64_t r = 0; r < n; ++r) {
      acc += (row_ptr[r + 1] - row_ptr[r]) + 2.0;
      if (m < G && acc >= total * (double)m / (double)G && r + 1 < n) g_plan.cta_row0[m++] = (int32_t)(r + 1);
    }
    while (m < G + 1) g_plan.cta_row0[m++] = (int32_t)n;
    int32_t maxch = 1;
    for (int64_t c = 0; c < G; ++c)
      maxch = std::max(maxch, g_plan.row_chunk0[g_plan.cta_row0[c + 1]] - g_plan.row_chunk0[g_plan.cta_row0[c]]);
    smem = sizeof(double) * 6 * (size_t)maxch;
    if (smem <= 48 * 1024 && pcg_occupancy_f64(smem) * (int64_t)sms >= G) break;
    if (G == 1 || smem > 48 * 1024) {
      set_msg(err, err_len, "ba_pcg_solve_static: rows too long for the kernel's shared-memory chunk buffer");
      return BA_ERR_ARG;
    }
    G = std::max<int64_t>(1, G / 2);
  }

  // inputs of the kernels into the scratch array; the scalars start at zero
  auto fail_cuda = [&](cudaError_t e) {
    cudaGetLastError();
    char m[256];
    std::snprintf(m, sizeof(m), "ba_pcg_solve_static: %s", cudaGetErrorString(e));
    set_msg(err, err_len, m);
    return BA_ERR_CUDA;
  };
  cudaError_t e;
  if ((e = cudaMemcpyAsync(W->row_ptr, row_ptr, sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, st))) return fail_cuda(e);
  if ((e = cudaMemcpyAsync(W->cta_row0, g_plan.cta_row0, sizeof(int32_t) * (G + 1), cudaMemcpyHostToDevice, st))) return fail_cuda(e);
  if ((e = cudaMemcpyAsync(W->row_chunk0, g_plan.row_chunk0, sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, st))) return fail_cuda(e);
  if ((e = cudaMemcpyAsync(W->chunk_beg, g_plan.chunk_beg, sizeof(int32_t) * (nch + 1), cudaMemcpyHostToDevice, st))) return fail_cuda(e);
  if ((e = cudaMemsetAsync(&W->S, 0, sizeof(DevScalars), st))) return fail_cuda(e);
  k_check_pattern<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(n, W->row_ptr, cols, &W->S);
  if ((e = cudaGetLastError())) return fail_cuda(e);
  int flags = 0;
  if ((e = cudaMemcpyAsync(&flags, &W->S.flags, sizeof(int), cudaMemcpyDeviceToHost, st))) return fail_cuda(e);
  if ((e = cudaStreamSynchronize(st))) return fail_cuda(e);
  if (flags) {
    set_msg(err, err_len, (flags & 16) ? "ba_pcg_solve_static: a column index is out of range"
                                       : "ba_pcg_solve_static: a block row has no diagonal block");
    return BA_ERR_ARG;
  }
  if ((e = launch_precond_raw_f64(st, n, W->row_ptr, cols, vals, W->Minv, &W->S))) return fail_cuda(e);
  // a diagonal block whose Cholesky factorisation failed: S is not positive definite, and CG is not defined
  if ((e = cudaMemcpyAsync(&flags, &W->S.flags, sizeof(int), cudaMemcpyDeviceToHost, st))) return fail_cuda(e);
  if ((e = cudaStreamSynchronize(st))) return fail_cuda(e);
  if (flags & 4) {
    set_msg(err, err_len, "ba_pcg_solve_static: a diagonal block is not positive definite");
    return BA_ERR_ARG;
  }
  if ((e = launch_pcg_raw_f64(st, (int)G, smem, n, cols, W->cta_row0, W->row_chunk0, W->chunk_beg, vals, W->Minv, b,
                              x, W->r, W->z, W->p, W->Ap, W->part, &W->S, rel_tol, max_iters)))
    return fail_cuda(e);
  DevScalars h;
  if ((e = cudaMemcpyAsync(&h, &W->S, sizeof(DevScalars), cudaMemcpyDeviceToHost, st))) return fail_cuda(e);
  if ((e = cudaStreamSynchronize(st))) return fail_cuda(e);
  if (h.flags & PCG_FLAG_TIMEOUT) {
    set_msg(err, err_len, "ba_pcg_solve_static: a grid barrier of the PCG kernel waited too long");
    return BA_ERR_TIMEOUT;
  }
  if (iters) *iters = h.iters;
  if (rel) *rel = h.bnorm2 > 0 ? std::sqrt(h.rr / h.bnorm2) : 0.0;
  set_msg(err, err_len, "");
  return BA_OK;
}
