// mgsa_qr_noalloc: the single-instance QR with its scratch in a static device
// array instead of handle-owned allocations (declared in mgsa.h).
//
// Who needs it: callers that may not allocate device memory -- code living
// under a memory manager that owns the whole GPU (a caching allocator, a
// server admitting work against a fixed budget) and latency-critical loops
// that cannot afford the device-wide synchronisation of cudaMalloc/cudaFree.
//
// The kernel is the same cooperative kernel mgsa_qr launches; only the
// source of its scratch differs.  The array below is module data: every GPU
// that loads the library holds it until the process exits.  Host code may not
// use its name as a device address (on the host it names a stand-in), so the
// first call in each CUDA context, with that context current, looks the
// address up with cudaGetSymbolAddress and sets the kernel's shared-memory
// limit.  Both belong to the context: after cudaDeviceReset (or whenever
// another context becomes current on the device) the module is loaded again,
// possibly elsewhere, and the attribute is gone.  So the set-up is keyed on
// the current context's unique id (cuCtxGetId, reached through the runtime's
// driver entry points; no link to the driver library), and redone when it
// changes.
#include <cuda.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "mgsa.h"
#include "mgsa_internal.cuh"

namespace {

constexpr size_t kScratchBytes = MGSA_NOALLOC_SCRATCH_BYTES;
constexpr size_t kCtlBytes = 256;  // status + barrier words, then padding
constexpr int kMaxDevices = 64;

// Layout of one call's scratch: [ctl: 256 B][per-CTA partials][x / p columns].
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_setup_mutex;
struct DeviceSetup {
  unsigned long long ctx_id = 0;  // id of the context the set-up was done in (0: none yet)
  void* addr = nullptr;           // device address of g_noalloc_scratch in that context
};
DeviceSetup g_setup[kMaxDevices];

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

int64_t round_up(int64_t x, int64_t q) { return (x + q - 1) / q * q; }

mgsa_status fail(mgsa_status s, const char* why) {
  mgsa::set_last_error(why);
  return s;
}

mgsa_status cuda_fail(cudaError_t e) {
  mgsa::set_last_error(cudaGetErrorString(e));
  return MGSA_ERR_CUDA;
}

// The unique id of the context current on this thread; when none is current
// yet, the device's primary context is initialised and made current first.
// Caller holds g_setup_mutex.
mgsa_status current_context_id(int dev, unsigned long long* id) {
  cudaError_t e = cudaSuccess;
  if (!g_ctx_get_current || !g_ctx_get_id) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = cudaDriverEntryPointSymbolNotFound;
    if ((e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1)) != cudaSuccess)
      return cuda_fail(e);
    if ((e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2)) != cudaSuccess)
      return cuda_fail(e);
    if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
      return fail(MGSA_ERR_CUDA, "the driver does not provide cuCtxGetCurrent / cuCtxGetId");
    g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
    g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f2);
  }
  CUcontext ctx = nullptr;
  if (g_ctx_get_current(&ctx) != CUDA_SUCCESS) return fail(MGSA_ERR_CUDA, "cuCtxGetCurrent failed");
  if (!ctx) {
    if ((e = cudaSetDevice(dev)) != cudaSuccess) return cuda_fail(e);
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx) return fail(MGSA_ERR_CUDA, "no current CUDA context");
  }
  if (g_ctx_get_id(ctx, id) != CUDA_SUCCESS) return fail(MGSA_ERR_CUDA, "cuCtxGetId failed");
  return MGSA_OK;
}

// Once per context, with that context current: the array's device address and
// the kernel's shared-memory attribute.  Later calls in the same context reuse
// them; a call in a new context (after cudaDeviceReset, say) repeats both.
mgsa_status device_setup(int dev, unsigned char** scratch) {
  if (dev < 0 || dev >= kMaxDevices) return fail(MGSA_ERR_INVALID, "device ordinal beyond the set-up table");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  unsigned long long id = 0;
  mgsa_status st = current_context_id(dev, &id);
  if (st != MGSA_OK) return st;
  DeviceSetup& d = g_setup[dev];
  if (d.ctx_id != id || !d.addr) {
    d.ctx_id = 0;
    d.addr = nullptr;
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e);
    if ((e = mgsa::sweep_prepare(dev)) != cudaSuccess) return cuda_fail(e);
    d.addr = p;
    d.ctx_id = id;
  }
  *scratch = static_cast<unsigned char*>(d.addr);
  return MGSA_OK;
}

bool overlap(const void* a, size_t an, const void* b, size_t bn) {
  const uintptr_t a0 = (uintptr_t)a, b0 = (uintptr_t)b;
  return a0 < b0 + bn && b0 < a0 + an;
}

}  // namespace

extern "C" mgsa_status mgsa_qr_noalloc(const mgsa_csr* A, const double* Z, int64_t m, int n, int64_t ldz,
                                       mgsa_variant v, double* Q, int64_t ldq, double* R, int ldr, int* info_dev,
                                       mgsa_stream_t s) {
  if (!A || !Z || !Q || !R) return fail(MGSA_ERR_INVALID, "NULL matrix pointer");
  if (n < 1 || n > MGSA_MAX_N) return fail(MGSA_ERR_INVALID, "n must be in [1, MGSA_MAX_N]");
  if (m < n || m >= ((int64_t)1 << 31)) return fail(MGSA_ERR_INVALID, "m must satisfy n <= m < 2^31");
  if (ldz < m || ldq < m || ldr < n) return fail(MGSA_ERR_INVALID, "leading dimension too small");
  if (v != MGSA_NAIVE && v != MGSA_HA && v != MGSA_HP) return fail(MGSA_ERR_INVALID, "unknown or CGS variant");
  if (A->m != m) return fail(MGSA_ERR_INVALID, "A->m differs from m");
  if (A->nnz < 0 || A->nnz >= ((int64_t)1 << 31)) return fail(MGSA_ERR_INVALID, "nnz must be in [0, 2^31)");
  if (!A->rowptr || (A->nnz > 0 && (!A->col || !A->val))) return fail(MGSA_ERR_INVALID, "NULL CSR array");
  const size_t zspan = sizeof(double) * (size_t)((n - 1) * ldz + m);
  const size_t qspan = sizeof(double) * (size_t)((n - 1) * ldq + m);
  const size_t rspan = sizeof(double) * (size_t)((int64_t)(n - 1) * ldr + n);
  const bool in_place = static_cast<const void*>(Q) == static_cast<const void*>(Z) && ldq == ldz;  // Q = Z allowed
  if ((!in_place && overlap(Z, zspan, Q, qspan)) || overlap(R, rspan, Q, qspan) || overlap(R, rspan, Z, zspan))
    return fail(MGSA_ERR_INVALID, "Q, R and Z must not overlap (Q may be Z itself)");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e);
  unsigned char* scratch = nullptr;
  mgsa_status st = device_setup(dev, &scratch);
  if (st != MGSA_OK) return st;

  // Launch shape: the defaults of mgsa_qr (one CTA per SM that fits, slabs of
  // at least kMinRowsPerCta rows -- kMinRowsLongRows for long rows -- and
  // pivot chunks of kMaxChunk rows).
  int max_ctas = 0;
  if ((e = mgsa::sweep_max_ctas((int)v, mgsa::sweep_smem_bytes(n, mgsa::kMaxChunk), &max_ctas)) != cudaSuccess)
    return cuda_fail(e);
  if (max_ctas < 1) return fail(MGSA_ERR_CUDA, "sweep kernel does not fit on this device");
  const int64_t min_rows =
      A->nnz >= (int64_t)mgsa::kWarpRowNnz * m ? mgsa::kMinRowsLongRows : mgsa::kMinRowsPerCta;
  int64_t g = std::min<int64_t>(max_ctas, (m + min_rows - 1) / min_rows);
  g = std::max<int64_t>(g, 1);
  const int64_t rpc = round_up((m + g - 1) / g, 32);
  const int grid = (int)((m + rpc - 1) / rpc);
  const int chunk = (int)std::min<int64_t>(mgsa::kMaxChunk, rpc);
  const size_t smem = mgsa::sweep_smem_bytes(n, chunk, mgsa::sweep_pivot_rows(rpc <= chunk, (int)v));
  const int64_t ldx = round_up(m, 32);
  const int xcols = v == MGSA_HP ? n : (v == MGSA_HA ? 1 : 2);
  const size_t part_bytes = (size_t)round_up((int64_t)sizeof(double) * (2 * n + 1) * grid, 256);
  const size_t x_bytes = sizeof(double) * (size_t)ldx * (size_t)xcols;
  if (kCtlBytes + part_bytes + x_bytes > kScratchBytes)
    return fail(MGSA_ERR_INVALID,
                "problem too large for mgsa_qr_noalloc: its scratch exceeds MGSA_NOALLOC_SCRATCH_BYTES (32 MiB); "
                "use mgsa_qr");

  mgsa::SweepArgs a;
  a.m = m;
  a.n = n;
  a.rowptr = A->rowptr;
  a.col = A->col;
  a.val = A->val;
  a.Z = Z;
  a.ldz = ldz;
  a.Q = Q;
  a.ldq = ldq;
  a.R = R;
  a.ldr = ldr;
  a.ctl = reinterpret_cast<int*>(scratch);
  a.part = reinterpret_cast<double*>(scratch + kCtlBytes);
  a.X = reinterpret_cast<double*>(scratch + kCtlBytes + part_bytes);
  a.ldx = ldx;
  a.rpc = rpc;
  a.chunk = chunk;
  a.mv_warp = A->nnz >= (int64_t)mgsa::kWarpRowNnz * m;

  cudaStream_t cs = reinterpret_cast<cudaStream_t>(s);
  // The status and barrier words must start at zero; the rest of the array is
  // written before it is read.
  if ((e = cudaMemsetAsync(a.ctl, 0, sizeof(int) * mgsa::kCtlWords, cs)) != cudaSuccess) return cuda_fail(e);
  if ((e = mgsa::sweep_launch((int)v, a, grid, smem, cs)) != cudaSuccess) return cuda_fail(e);
  if (info_dev && (e = cudaMemcpyAsync(info_dev, a.ctl, 2 * sizeof(int), cudaMemcpyDeviceToDevice, cs)) != cudaSuccess)
    return cuda_fail(e);
  return MGSA_OK;
}
