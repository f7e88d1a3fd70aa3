// C-ABI of libmgsa: handle, argument checks, workspace and launches.
// The numerical work is done by the kernels in mgsa_sweep.cu.
#include <algorithm>
#include <cstddef>
#include <cstring>
#include <utility>

#include "mgsa.h"
#include "mgsa_internal.cuh"

struct mgsa_context {
  int device = 0;
  int* ctl = nullptr;          // device control block (status word, barrier state)
  int* ctl_host = nullptr;     // pinned mirror read by mgsa_get_info
  double* ws = nullptr;        // X columns + per-CTA partials
  size_t ws_bytes = 0;
  unsigned char* io = nullptr; // device staging of mgsa_qr_host
  size_t io_bytes = 0;
  int64_t max_ctas = 0;        // MGSA_PARAM_MAX_CTAS (0 = co-resident maximum)
  int chunk_rows = 0;          // MGSA_PARAM_CHUNK_ROWS (0 = kMaxChunk)
  int64_t min_rows = 0;        // MGSA_PARAM_MIN_ROWS_PER_CTA (0 = kMinRowsPerCta)
  double* batch_scratch = nullptr;  // per-CTA partial sums of the batched kernels
  int batch_grid = 0;               // CTAs of a batched launch (co-resident maximum)
  int64_t batch_ctas = 0;           // MGSA_PARAM_BATCH_CTAS (0 = batch_grid)
  int row_mode = 0;                 // MGSA_PARAM_ROW_MODE
  int spmm_panel = 8;               // MGSA_PARAM_SPMM_PANEL
  int cluster = 0;                  // MGSA_PARAM_CLUSTER: 0 auto, 1 never, c >= 2 a cluster of c CTAs
  bool wait_fault = false;          // MGSA_PARAM_WAIT_FAULT: first device-wide wait one arrival short
  size_t batch_smem = 0;
};

static_assert(sizeof(mgsa_job) == sizeof(mgsa::BatchJob), "mgsa_job and BatchJob must match");
static_assert(offsetof(mgsa_job, work) == offsetof(mgsa::BatchJob, work), "mgsa_job and BatchJob must match");

namespace {

thread_local const char* g_last_error = "no error";

mgsa_status fail(mgsa_status s, const char* why) {
  g_last_error = why;
  return s;
}

mgsa_status cuda_fail(cudaError_t e) {
  g_last_error = cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? MGSA_ERR_NOMEM : MGSA_ERR_CUDA;
}

// Restores the caller's current device on scope exit.
struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) return;
    ok = (prev == dev) || cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    if (ok && prev >= 0) {
      int cur = -1;
      if (cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
  }
};

int64_t round_up(int64_t x, int64_t q) { return (x + q - 1) / q * q; }

constexpr int64_t kBatchStride = 2 * mgsa::kBatchMaxN + 8;  // doubles of partial sums per batched CTA
constexpr int kBatchQueueWord = 16;                        // ctl[16..18]: batched job queues

struct Plan {
  int grid = 1;
  int64_t rpc = 32;
  int chunk = 32;
  size_t smem = 0;
  int64_t ldx = 0;
  int xcols = 0;
  size_t x_bytes = 0;
  size_t part_bytes = 0;
  int stages = 0;          // CGS: pivot buffers in shared memory
  int64_t qp_doubles = 0;  // CGS: pivot blocks (inside x_bytes, after the X columns)
  bool cluster = false;    // one thread-block cluster of `grid` CTAs instead of a cooperative grid
};

// nnz < 0: unknown (workspace sizing); long rows (warp-per-row MVs) carry
// more work per row, so they get smaller slabs and thus more CTAs.  kg given
// columns in front (successive orthogonalisation) widen the shared rows and
// partial sums to kg + n columns; the X columns stay those of the n new ones.
bool is_cgs(mgsa_variant v) { return v == MGSA_CGS_NAIVE || v == MGSA_CGS_HA || v == MGSA_CGS_HP; }

// Kernel template index (naive / HA / HP) of a public variant.
int kernel_variant(mgsa_variant v) { return is_cgs(v) ? (int)v - 3 : (int)v; }

constexpr int kCgsStagedChunk = 2048;  // CGS slabs above one chunk: rows per streamed chunk

// Shared memory of a plan (and, for CGS, the number of pivot buffers).
// piv_rows: pivot rows per chunk row of the MGS kernel (4 covers every slab).
mgsa_status plan_smem(mgsa_variant v, int nt, int chunk, size_t* smem, int* stages, int piv_rows = 4) {
  *stages = 0;
  if (!is_cgs(v)) {
    *smem = mgsa::sweep_smem_bytes(nt, chunk, piv_rows);
    return MGSA_OK;
  }
  cudaError_t e = mgsa::cgs_smem_plan(kernel_variant(v), nt, chunk, stages, smem);
  if (e == cudaErrorInvalidValue) return fail(MGSA_ERR_INVALID, "n too large for the CGS kernel's shared memory");
  return e == cudaSuccess ? MGSA_OK : cuda_fail(e);
}

mgsa_status make_plan(const mgsa_context* h, int64_t m, int n, mgsa_variant v, Plan* p, int64_t nnz = -1,
                      int kg = 0, bool allow_cluster = true) {
  const int nt = kg + n;
  const int chunk_cap = h->chunk_rows > 0 ? h->chunk_rows : mgsa::kMaxChunk;
  const bool long_rows = h->row_mode == 0 ? nnz >= (int64_t)mgsa::kWarpRowNnz * m : h->row_mode == 2;
  const int64_t min_rows = h->min_rows > 0 ? h->min_rows : (long_rows ? mgsa::kMinRowsLongRows : mgsa::kMinRowsPerCta);
  int max_ctas = 0;
  const int kv = kernel_variant(v);
  size_t smem_cap = 0;
  int stages = 0;
  mgsa_status st = plan_smem(v, nt, chunk_cap, &smem_cap, &stages);
  if (st != MGSA_OK) return st;
  cudaError_t e = is_cgs(v) ? mgsa::cgs_max_ctas(kv, smem_cap, &max_ctas) : mgsa::sweep_max_ctas(kv, smem_cap, &max_ctas);
  if (e != cudaSuccess) return cuda_fail(e);
  if (max_ctas < 1) return fail(MGSA_ERR_CUDA, "sweep kernel does not fit on this device");
  int64_t g = std::min<int64_t>(max_ctas, (m + min_rows - 1) / min_rows);
  if (h->max_ctas > 0) g = std::min<int64_t>(g, h->max_ctas);
  g = std::max<int64_t>(g, 1);
  // One thread-block cluster (hardware barriers) for small problems: its
  // barriers are ~0.5 us cheaper each, three or four per step, and it leaves
  // the FP64 rate of the other SMs unused.  On GB300 a 16-CTA cluster is
  // 12% faster than the grid at m = 1024, 1-3% at m = 4096 (n = 16 .. 64) and
  // slower from m = 8192 up, so: at most 256 rows per CTA and m (k + n) <= 2^18.
  // Not for CGS or time slices (cooperative kernels only).
  p->cluster = false;
  if (!is_cgs(v) && allow_cluster && h->cluster != 1) {
    int cmax = 0;
    if ((e = mgsa::cluster_max_size(kv, smem_cap, &cmax)) != cudaSuccess) return cuda_fail(e);
    const int want = h->cluster >= 2 ? h->cluster : cmax;
    const bool small = m * (int64_t)nt <= ((int64_t)1 << 18) && m <= (int64_t)want * 256;
    if (want >= 1 && want <= cmax && (h->cluster >= 2 || small)) {
      p->cluster = true;
      g = want;
    } else if (h->cluster >= 2) {
      return fail(MGSA_ERR_INVALID, "cluster size above what the GPU can co-schedule");
    }
  }
  p->rpc = round_up((m + g - 1) / g, 32);
  p->grid = (int)((m + p->rpc - 1) / p->rpc);
  p->chunk = (int)std::min<int64_t>(chunk_cap, p->rpc);
  // CGS streams a slab that is not one chunk in smaller chunks, so that more
  // pivot buffers fit in shared memory.
  if (is_cgs(v) && p->rpc > chunk_cap && h->chunk_rows == 0) p->chunk = kCgsStagedChunk;
  const int piv_rows = mgsa::sweep_pivot_rows(p->rpc <= p->chunk, kv);  // the layout the kernel takes
  if ((st = plan_smem(v, nt, p->chunk, &p->smem, &p->stages, piv_rows)) != MGSA_OK) return st;
  p->ldx = round_up(m, 32);
  if (is_cgs(v)) p->xcols = v == MGSA_CGS_HP ? n : 2;
  else p->xcols = v == MGSA_HP ? n : (v == MGSA_HA ? 1 : 2);
  // CGS pivot blocks: 2 * n * G * rpc doubles, and G * rpc <= m + 32 * G for
  // every grid G a plan can choose, so a reservation fits every nnz.
  const int64_t gmax = std::max<int64_t>(max_ctas, p->grid);
  p->qp_doubles = is_cgs(v) ? 2 * (int64_t)n * (p->ldx + 32 * gmax) : 0;
  p->x_bytes = (size_t)round_up((int64_t)sizeof(double) * (p->ldx * p->xcols + p->qp_doubles), 256);
  // Partials for the largest grid any plan can use, so a reservation fits every nnz.
  p->part_bytes = sizeof(double) * (size_t)(2 * nt + 1) * (size_t)gmax;
  return MGSA_OK;
}

mgsa_status ensure_ws(mgsa_handle h, size_t bytes) {
  if (bytes <= h->ws_bytes) return MGSA_OK;
  if (h->ws) {
    cudaError_t e = cudaFree(h->ws);
    h->ws = nullptr;
    h->ws_bytes = 0;
    if (e != cudaSuccess) return cuda_fail(e);
  }
  cudaError_t e = cudaMalloc(&h->ws, bytes);
  if (e != cudaSuccess) return cuda_fail(e);
  h->ws_bytes = bytes;
  return MGSA_OK;
}

bool ranges_overlap(const void* a, size_t an, const void* b, size_t bn) {
  const uintptr_t a0 = (uintptr_t)a, b0 = (uintptr_t)b;
  return a0 < b0 + bn && b0 < a0 + an;
}

mgsa_status check_sizes(int64_t m, int n, int64_t ldz, mgsa_variant v, int64_t ldq, int ldr) {
  if (n < 1 || n > MGSA_MAX_N) return fail(MGSA_ERR_INVALID, "n must be in [1, MGSA_MAX_N]");
  if (m < n || m >= ((int64_t)1 << 31)) return fail(MGSA_ERR_INVALID, "m must satisfy n <= m < 2^31");
  if (ldz < m || ldq < m) return fail(MGSA_ERR_INVALID, "leading dimension of Z or Q below m");
  if (ldr < n) return fail(MGSA_ERR_INVALID, "leading dimension of R below n");
  if ((int)v < (int)MGSA_NAIVE || (int)v > (int)MGSA_CGS_HP) return fail(MGSA_ERR_INVALID, "unknown variant");
  return MGSA_OK;
}

}  // namespace

// Lets other translation units of the library report through mgsa_last_error.
void mgsa::set_last_error(const char* why) { g_last_error = why; }

extern "C" {

const char* mgsa_last_error(void) { return g_last_error; }

mgsa_status mgsa_create(mgsa_handle* h, int device) {
  if (!h) return fail(MGSA_ERR_INVALID, "NULL handle pointer");
  *h = nullptr;
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess) return cuda_fail(e);
  if (device < 0 || device >= count) return fail(MGSA_ERR_INVALID, "no such CUDA device");
  DeviceGuard g(device);
  if (!g.ok) return fail(MGSA_ERR_CUDA, "cannot select the device");
  mgsa_context* c = new (std::nothrow) mgsa_context;
  if (!c) return fail(MGSA_ERR_NOMEM, "host allocation failed");
  c->device = device;
  if ((e = cudaMalloc(&c->ctl, 256)) != cudaSuccess || (e = cudaMemset(c->ctl, 0, 256)) != cudaSuccess ||
      (e = cudaMallocHost(&c->ctl_host, 256)) != cudaSuccess || (e = mgsa::sweep_prepare(device)) != cudaSuccess ||
      (e = mgsa::cgs_prepare(device)) != cudaSuccess || (e = mgsa::cluster_prepare(device)) != cudaSuccess) {
    mgsa_status s = cuda_fail(e);
    mgsa_destroy(c);
    return s;
  }
  // Batched kernels: shared memory for n <= kBatchMaxN, one CTA per SM that fits,
  // and their per-CTA partial sums (allocated here so mgsa_qr_batched never allocates).
  c->batch_smem = mgsa::sweep_smem_bytes(mgsa::kBatchMaxN, mgsa::kMaxChunk);
  if ((e = mgsa::batch_prepare(device, c->batch_smem)) != cudaSuccess ||
      (e = mgsa::batch_max_ctas(c->batch_smem, &c->batch_grid)) != cudaSuccess ||
      (e = cudaMalloc(&c->batch_scratch, sizeof(double) * (size_t)c->batch_grid * kBatchStride)) != cudaSuccess) {
    mgsa_status s = cuda_fail(e);
    mgsa_destroy(c);
    return s;
  }
  std::memset(c->ctl_host, 0, 256);
  *h = c;
  return MGSA_OK;
}

mgsa_status mgsa_destroy(mgsa_handle h) {
  if (!h) return MGSA_OK;
  {
    DeviceGuard g(h->device);
    if (h->ws) cudaFree(h->ws);
    if (h->io) cudaFree(h->io);
    if (h->batch_scratch) cudaFree(h->batch_scratch);
    if (h->ctl) cudaFree(h->ctl);
    if (h->ctl_host) cudaFreeHost(h->ctl_host);
  }
  delete h;
  return MGSA_OK;
}

size_t mgsa_workspace_bytes(mgsa_handle h, int64_t m, int n, mgsa_variant v) {
  if (!h || check_sizes(m, n, m, v, m, n) != MGSA_OK) return 0;
  DeviceGuard g(h->device);
  Plan p;
  if (make_plan(h, m, n, v, &p) != MGSA_OK) return 0;
  return p.x_bytes + p.part_bytes;
}

mgsa_status mgsa_reserve(mgsa_handle h, int64_t m, int n, mgsa_variant v) {
  if (!h) return fail(MGSA_ERR_INVALID, "NULL handle");
  mgsa_status s = check_sizes(m, n, m, v, m, n);
  if (s != MGSA_OK) return s;
  DeviceGuard g(h->device);
  if (!g.ok) return fail(MGSA_ERR_CUDA, "cannot select the device");
  Plan p;
  if ((s = make_plan(h, m, n, v, &p)) != MGSA_OK) return s;
  return ensure_ws(h, p.x_bytes + p.part_bytes);
}

mgsa_status mgsa_set_param(mgsa_handle h, mgsa_param p, int64_t value) {
  if (!h) return fail(MGSA_ERR_INVALID, "NULL handle");
  if (value < 0) return fail(MGSA_ERR_INVALID, "parameter value must be >= 0");
  switch (p) {
    case MGSA_PARAM_MAX_CTAS: h->max_ctas = value; return MGSA_OK;
    case MGSA_PARAM_CHUNK_ROWS:
      if (value % 32 != 0 || value > mgsa::kMaxChunk) return fail(MGSA_ERR_INVALID, "chunk rows: multiple of 32, <= 4096");
      h->chunk_rows = (int)value;
      return MGSA_OK;
    case MGSA_PARAM_MIN_ROWS_PER_CTA: h->min_rows = value; return MGSA_OK;
    case MGSA_PARAM_BATCH_CTAS: h->batch_ctas = value; return MGSA_OK;
    case MGSA_PARAM_ROW_MODE:
      if (value > 2) return fail(MGSA_ERR_INVALID, "row mode: 0 (auto), 1 (thread per row) or 2 (warp per row)");
      h->row_mode = (int)value;
      return MGSA_OK;
    case MGSA_PARAM_CLUSTER:
      if (value > mgsa::kMaxClusterCtas) return fail(MGSA_ERR_INVALID, "cluster: 0 (auto), 1 (never) or 2..16 CTAs");
      h->cluster = (int)value;
      return MGSA_OK;
    case MGSA_PARAM_SPMM_PANEL:
      if (value != 0 && value != 4 && value != 8) return fail(MGSA_ERR_INVALID, "SpMM panel: 0 (default 8), 4 or 8");
      h->spmm_panel = value == 0 ? 8 : (int)value;
      return MGSA_OK;
    case MGSA_PARAM_WAIT_FAULT:
      if (value > 1) return fail(MGSA_ERR_INVALID, "wait fault: 0 (off) or 1 (on)");
      h->wait_fault = value == 1;
      return MGSA_OK;
    default: return fail(MGSA_ERR_INVALID, "unknown parameter");
  }
}

// Checks shared by mgsa_qr and mgsa_qr_append, then one cooperative launch.
// kg given columns Qg (with their p_i in Pg) precede the n columns of Z; P
// (nullable) receives the p_j of the new columns.
static mgsa_status qr_launch(mgsa_handle h, const mgsa_csr* A, const double* Z, int64_t m, int n, int64_t ldz,
                             mgsa_variant v, double* Q, int64_t ldq, double* R, int ldr, int kg, const double* Qg,
                             int64_t ldqg, const double* Pg, int64_t ldpg, double* P, int64_t ldp, mgsa_stream_t s,
                             int step_begin = 0, int step_end = -1) {
  if (!h) return fail(MGSA_ERR_INVALID, "NULL handle");
  if (!A || !Z || !Q || !R) return fail(MGSA_ERR_INVALID, "NULL matrix pointer");
  if (kg < 0 || kg > MGSA_MAX_N - 1) return fail(MGSA_ERR_INVALID, "k must be in [0, MGSA_MAX_N)");
  mgsa_status st = check_sizes(m, n, ldz, v, ldq, n);  // ldr is checked against k + n below
  if (st != MGSA_OK) return st;
  if (is_cgs(v) && (kg > 0 || P)) return fail(MGSA_ERR_INVALID, "the CGS variants take no given columns and no P");
  const int nt = kg + n;
  if (nt > MGSA_MAX_N) return fail(MGSA_ERR_INVALID, "k + n must be <= MGSA_MAX_N");
  if (m < nt) return fail(MGSA_ERR_INVALID, "m must be >= k + n");
  if (ldr < nt) return fail(MGSA_ERR_INVALID, "leading dimension of R below k + n");
  if (kg > 0) {
    if (!Qg || !Pg) return fail(MGSA_ERR_INVALID, "NULL given Q or P");
    if (ldqg < m || ldpg < m) return fail(MGSA_ERR_INVALID, "leading dimension of the given Q or P below m");
  }
  if (P && ldp < m) return fail(MGSA_ERR_INVALID, "leading dimension of P below m");
  if (A->m != m) return fail(MGSA_ERR_INVALID, "A->m differs from m");
  if (A->nnz < 0 || A->nnz >= ((int64_t)1 << 31)) return fail(MGSA_ERR_INVALID, "nnz must be in [0, 2^31)");
  if (!A->rowptr || (A->nnz > 0 && (!A->col || !A->val))) return fail(MGSA_ERR_INVALID, "NULL CSR array");
  const size_t zspan = sizeof(double) * (size_t)((n - 1) * ldz + m);
  const size_t qspan = sizeof(double) * (size_t)((n - 1) * ldq + m);
  // Q may be Z itself (same pointer and leading dimension): the kernels read
  // Z only before their first device-wide wait, or only columns they have not
  // yet written.  Any other overlap is refused.
  const bool in_place = static_cast<const void*>(Q) == static_cast<const void*>(Z) && ldq == ldz;
  if (!in_place && ranges_overlap(Z, zspan, Q, qspan)) return fail(MGSA_ERR_INVALID, "Q overlaps Z");
  const size_t rspan = sizeof(double) * (size_t)((int64_t)(n - 1) * ldr + nt);
  if (ranges_overlap(R, rspan, Q, qspan) || ranges_overlap(R, rspan, Z, zspan))
    return fail(MGSA_ERR_INVALID, "R overlaps Q or Z");
  const size_t pspan = P ? sizeof(double) * (size_t)((n - 1) * ldp + m) : 0;
  if (P && (ranges_overlap(P, pspan, Q, qspan) || ranges_overlap(P, pspan, Z, zspan) ||
            ranges_overlap(P, pspan, R, rspan)))
    return fail(MGSA_ERR_INVALID, "P overlaps Q, Z or R");
  if (kg > 0) {
    const size_t gq = sizeof(double) * (size_t)((kg - 1) * ldqg + m);
    const size_t gp = sizeof(double) * (size_t)((kg - 1) * ldpg + m);
    for (const auto& o : {std::make_pair((const void*)Q, qspan), std::make_pair((const void*)R, rspan),
                          std::make_pair((const void*)P, pspan)})
      if (o.second && (ranges_overlap(Qg, gq, o.first, o.second) || ranges_overlap(Pg, gp, o.first, o.second)))
        return fail(MGSA_ERR_INVALID, "an output overlaps the given Q or P");
  }

  DeviceGuard g(h->device);
  if (!g.ok) return fail(MGSA_ERR_CUDA, "cannot select the device");
  Plan p;
  const bool sliced = step_begin != 0 || step_end >= 0;
  if ((st = make_plan(h, m, n, v, &p, A->nnz, kg, !sliced)) != MGSA_OK) return st;
  if ((st = ensure_ws(h, p.x_bytes + p.part_bytes)) != MGSA_OK) return st;

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
  a.X = h->ws;
  a.ldx = p.ldx;
  a.part = reinterpret_cast<double*>(reinterpret_cast<unsigned char*>(h->ws) + p.x_bytes);
  a.ctl = h->ctl;
  a.rpc = p.rpc;
  a.chunk = p.chunk;
  a.mv_warp = h->row_mode == 0 ? A->nnz >= (int64_t)mgsa::kWarpRowNnz * m : h->row_mode == 2;
  a.spmm_panel = h->spmm_panel;
  if (is_cgs(v)) {
    a.qp = a.X + p.ldx * p.xcols;
    a.stages = p.stages;
  }
  a.step_begin = step_begin;
  a.step_end = step_end;
  a.kg = kg;
  a.Qg = Qg;
  a.ldqg = ldqg;
  a.Pg = Pg;
  a.ldpg = ldpg;
  if (P && v == MGSA_HP) {
    a.X = P;  // HP keeps x_j, then p_j, in X: let them land in P directly
    a.ldx = ldp;
  } else {
    a.Pout = P;
    a.ldpo = ldp;
  }

  cudaStream_t cs = reinterpret_cast<cudaStream_t>(s);
  // A first slice clears the whole control block; a later one only the
  // barrier counters (the status word carries an earlier slice's failure).
  cudaError_t e = step_begin == 0 ? cudaMemsetAsync(h->ctl, 0, sizeof(int) * mgsa::kCtlWords, cs)
                                  : cudaMemsetAsync(h->ctl + mgsa::kCtlBarCount, 0, 2 * sizeof(int), cs);
  if (e != cudaSuccess) return cuda_fail(e);
  // Failure-detection test hook: with the counter at 2^32 - 1 the first
  // barrier's arrivals wrap it to grid - 1, one short of its target grid, so
  // every CTA's bounded wait runs out (each CTA reads the counter only after
  // its own arrival, never the initial value).
  if (h->wait_fault && !is_cgs(v) && !p.cluster &&
      (e = cudaMemsetAsync(h->ctl + mgsa::kCtlBarCount, 0xFF, sizeof(int), cs)) != cudaSuccess)
    return cuda_fail(e);
  if (is_cgs(v)) e = mgsa::cgs_launch(kernel_variant(v), a, p.grid, p.smem, cs);
  else if (p.cluster) e = mgsa::cluster_launch(kernel_variant(v), a, p.grid, p.smem, cs);
  else e = mgsa::sweep_launch(kernel_variant(v), a, p.grid, p.smem, cs);
  if (e != cudaSuccess) return cuda_fail(e);
  return MGSA_OK;
}

mgsa_status mgsa_qr(mgsa_handle h, const mgsa_csr* A, const double* Z, int64_t m, int n, int64_t ldz,
                    mgsa_variant v, double* Q, int64_t ldq, double* R, int ldr, mgsa_stream_t s) {
  return qr_launch(h, A, Z, m, n, ldz, v, Q, ldq, R, ldr, 0, nullptr, 0, nullptr, 0, nullptr, 0, s);
}

mgsa_status mgsa_qr_steps(mgsa_handle h, const mgsa_csr* A, const double* Z, int64_t m, int n, int64_t ldz,
                          mgsa_variant v, double* Q, int64_t ldq, double* R, int ldr, int first, int count,
                          mgsa_stream_t s) {
  if (v != MGSA_NAIVE && v != MGSA_HA && v != MGSA_HP) return fail(MGSA_ERR_INVALID, "time slicing takes MGS forms only");
  if (first < 0 || count < 1 || first >= n || count > n - first)
    return fail(MGSA_ERR_INVALID, "steps [first, first + count) must lie in [0, n)");
  return qr_launch(h, A, Z, m, n, ldz, v, Q, ldq, R, ldr, 0, nullptr, 0, nullptr, 0, nullptr, 0, s, first,
                   first + count);
}

mgsa_status mgsa_qr_append(mgsa_handle h, const mgsa_csr* A, const double* Qold, int64_t ldqo, const double* Pold,
                           int64_t ldpo, int k, const double* Z, int64_t m, int n, int64_t ldz, mgsa_variant v,
                           double* Q, int64_t ldq, double* P, int64_t ldp, double* R, int ldr, mgsa_stream_t s) {
  if (is_cgs(v)) return fail(MGSA_ERR_INVALID, "mgsa_qr_append takes the MGS variants only");
  return qr_launch(h, A, Z, m, n, ldz, v, Q, ldq, R, ldr, k, Qold, ldqo, Pold, ldpo, P, ldp, s);
}

size_t mgsa_job_workspace_bytes(int64_t m, int n, mgsa_variant v) {
  if (m < 1 || n < 1 || (v != MGSA_NAIVE && v != MGSA_HA && v != MGSA_HP)) return 0;
  const int64_t cols = v == MGSA_HP ? n : (v == MGSA_HA ? 1 : 2);
  return sizeof(double) * (size_t)round_up(m, 32) * (size_t)cols;
}

mgsa_status mgsa_qr_batched(mgsa_handle h, int count, const mgsa_job* jobs_dev, int* info_dev, mgsa_stream_t s) {
  if (!h) return fail(MGSA_ERR_INVALID, "NULL handle");
  if (count < 0) return fail(MGSA_ERR_INVALID, "count must be >= 0");
  if (count == 0) return MGSA_OK;
  if (!jobs_dev || !info_dev) return fail(MGSA_ERR_INVALID, "NULL job or info array");
  DeviceGuard g(h->device);
  if (!g.ok) return fail(MGSA_ERR_CUDA, "cannot select the device");
  mgsa::BatchArgs ba;
  ba.jobs = reinterpret_cast<const mgsa::BatchJob*>(jobs_dev);
  ba.count = count;
  ba.max_n = mgsa::kBatchMaxN;
  ba.info = info_dev;
  ba.queue = reinterpret_cast<unsigned int*>(h->ctl + kBatchQueueWord);
  ba.scratch = h->batch_scratch;
  ba.scratch_stride = kBatchStride;
  ba.row_mode = h->row_mode;
  ba.spmm_panel = h->spmm_panel;
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(s);
  cudaError_t e = cudaMemsetAsync(ba.queue, 0, 3 * sizeof(unsigned int), cs);
  const int grid = h->batch_ctas > 0 ? (int)std::min<int64_t>(h->batch_ctas, h->batch_grid) : h->batch_grid;
  if (e == cudaSuccess) e = mgsa::batch_launch(ba, grid, h->batch_smem, cs);
  if (e != cudaSuccess) return cuda_fail(e);
  return MGSA_OK;
}

// Grouped launch: per-CTA partials reserved for the most CTAs the device can
// ever hold at once (the smallest shared-memory footprint), so that a member
// may get a different gang size in each slice and its X columns sit at the
// same place in its workspace whatever the launch.
static int group_part_ctas(int* max_ctas) {
  int mc = 0;
  if (mgsa::group_max_ctas((int)MGSA_HP, mgsa::sweep_smem_bytes(1, 32), &mc) != cudaSuccess || mc < 1) return 0;
  *max_ctas = mc;
  return mc;
}

size_t mgsa_group_workspace_bytes(mgsa_handle h, int64_t m, int n, mgsa_variant v) {
  if (!h || m < 1 || n < 1 || n > MGSA_MAX_N || (v != MGSA_NAIVE && v != MGSA_HA && v != MGSA_HP)) return 0;
  DeviceGuard g(h->device);
  int mc = 0;
  if (!group_part_ctas(&mc)) return 0;
  const int64_t cols = v == MGSA_HP ? n : (v == MGSA_HA ? 1 : 2);
  return (size_t)mgsa::kGroupCtlBytes +
         (size_t)round_up(8 * mgsa::group_part_doubles(n, mc), 256) + sizeof(double) * (size_t)round_up(m, 32) * (size_t)cols;
}

mgsa_status mgsa_qr_group(mgsa_handle h, mgsa_variant v, int count, const mgsa_group_member* members,
                          mgsa_stream_t s) {
  if (!h) return fail(MGSA_ERR_INVALID, "NULL handle");
  if (v != MGSA_NAIVE && v != MGSA_HA && v != MGSA_HP) return fail(MGSA_ERR_INVALID, "grouped launches take MGS forms only");
  if (count < 1 || count > MGSA_GROUP_MAX) return fail(MGSA_ERR_INVALID, "count must be in [1, MGSA_GROUP_MAX]");
  if (!members) return fail(MGSA_ERR_INVALID, "NULL member array");
  DeviceGuard g(h->device);
  if (!g.ok) return fail(MGSA_ERR_CUDA, "cannot select the device");
  int max_n = 1;
  for (int k = 0; k < count; ++k) max_n = std::max(max_n, (int)members[k].job.n);
  if (max_n > MGSA_MAX_N) return fail(MGSA_ERR_INVALID, "n must be in [1, MGSA_MAX_N]");
  int mc = 0;
  if (!group_part_ctas(&mc)) return fail(MGSA_ERR_CUDA, "sweep kernel does not fit on this device");
  const int chunk_cap = h->chunk_rows > 0 ? h->chunk_rows : mgsa::kMaxChunk;
  static_assert(sizeof(mgsa::GroupArgs) <= 16 * 1024, "grouped launch arguments too large");
  mgsa::GroupArgs* ga = new (std::nothrow) mgsa::GroupArgs();
  if (!ga) return fail(MGSA_ERR_NOMEM, "host allocation failed");
  ga->count = count;
  ga->spmm_panel = h->spmm_panel;
  int total = 0, chunk_max = 32;
  mgsa_status st = MGSA_OK;
  for (int k = 0; k < count && st == MGSA_OK; ++k) {
    const mgsa_group_member& M = members[k];
    const mgsa_job& J = M.job;
    if (J.variant != (int)v) st = fail(MGSA_ERR_INVALID, "a member's variant differs from the launch's");
    else if (check_sizes(J.m, J.n, J.ldz, v, J.ldq, (int)std::min<int64_t>(J.ldr, INT32_MAX)) != MGSA_OK) st = MGSA_ERR_INVALID;
    else if (!J.rowptr || !J.Z || !J.Q || !J.R || !J.work) st = fail(MGSA_ERR_INVALID, "NULL member pointer");
    else if ((reinterpret_cast<uintptr_t>(J.work) & 255) != 0) st = fail(MGSA_ERR_INVALID, "member workspace not 256-byte aligned");
    else if (M.first < 0 || M.count < 1 || M.first >= J.n || M.count > J.n - M.first)
      st = fail(MGSA_ERR_INVALID, "member steps [first, first + count) must lie in [0, n)");
    else if (M.ctas < 1) st = fail(MGSA_ERR_INVALID, "member ctas must be >= 1");
    for (int k2 = 0; k2 < k && st == MGSA_OK; ++k2)
      if (members[k2].job.work == J.work || members[k2].job.Q == J.Q || members[k2].job.R == J.R)
        st = fail(MGSA_ERR_INVALID, "two members share a workspace, Q or R");
    if (st != MGSA_OK) break;
    // The plan mgsa_qr would choose with MGSA_PARAM_MAX_CTAS = ctas and no
    // cluster.  The host does not read A, so the smallest slab is
    // kMinRowsPerCta unless the row mode says the rows are long; with the
    // automatic row mode the kernel reads nnz = rowptr[m] to pick the MV form.
    const bool long_rows = h->row_mode == 2;
    const int64_t min_rows = h->min_rows > 0 ? h->min_rows : (long_rows ? mgsa::kMinRowsLongRows : mgsa::kMinRowsPerCta);
    int64_t gk = std::min<int64_t>({(int64_t)M.ctas, (int64_t)mc, (J.m + min_rows - 1) / min_rows});
    gk = std::max<int64_t>(gk, 1);
    const int64_t rpc = round_up((J.m + gk - 1) / gk, 32);
    mgsa::GroupMember& D = ga->members[k];
    std::memcpy(&D.job, &J, sizeof(mgsa::BatchJob));
    D.first = M.first;
    D.count = M.count;
    D.rpc = (int)rpc;
    D.G = (int)((J.m + rpc - 1) / rpc);
    D.chunk = (int)std::min<int64_t>(chunk_cap, rpc);
    D.mv_warp = h->row_mode == 0 ? -1 : (h->row_mode == 2 ? 1 : 0);
    D.part_doubles = round_up(8 * mgsa::group_part_doubles(J.n, mc), 256) / 8;
    ga->offsets[k] = total;
    total += D.G;
    chunk_max = std::max(chunk_max, D.chunk);
  }
  const size_t smem = mgsa::sweep_smem_bytes(max_n, chunk_max);
  int cap = 0;
  if (st == MGSA_OK && mgsa::group_max_ctas((int)v, smem, &cap) != cudaSuccess)
    st = fail(MGSA_ERR_CUDA, "occupancy query failed");
  if (st == MGSA_OK && total > cap) st = fail(MGSA_ERR_INVALID, "the members' CTAs exceed what the GPU holds at once");
  if (st == MGSA_OK) {
    ga->offsets[count] = total;
    cudaError_t e = mgsa::group_launch((int)v, *ga, smem, reinterpret_cast<cudaStream_t>(s));
    if (e != cudaSuccess) st = cuda_fail(e);
  }
  delete ga;
  return st;
}

mgsa_status mgsa_copy_info(mgsa_handle h, int* info_dev, mgsa_stream_t s) {
  if (!h || !info_dev) return fail(MGSA_ERR_INVALID, "NULL handle or info_dev");
  DeviceGuard g(h->device);
  if (!g.ok) return fail(MGSA_ERR_CUDA, "cannot select the device");
  cudaError_t e = cudaMemcpyAsync(info_dev, h->ctl, 2 * sizeof(int), cudaMemcpyDeviceToDevice,
                                  reinterpret_cast<cudaStream_t>(s));
  return e == cudaSuccess ? MGSA_OK : cuda_fail(e);
}

mgsa_status mgsa_get_info(mgsa_handle h, mgsa_stream_t s, int* info) {
  if (!h || !info) return fail(MGSA_ERR_INVALID, "NULL handle or info");
  DeviceGuard g(h->device);
  if (!g.ok) return fail(MGSA_ERR_CUDA, "cannot select the device");
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(s);
  cudaError_t e = cudaMemcpyAsync(h->ctl_host, h->ctl, sizeof(int) * 2, cudaMemcpyDeviceToHost, cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
  if (e != cudaSuccess) return cuda_fail(e);
  const int code = h->ctl_host[mgsa::kCtlStatus];
  const int col = h->ctl_host[mgsa::kCtlColumn];
  switch (code) {
    case mgsa::kDevOk: *info = 0; return MGSA_OK;
    case mgsa::kDevBreakdown: *info = col; return fail(MGSA_ERR_BREAKDOWN, "z_j^T A z_j not positive");
    case mgsa::kDevNonfinite: *info = col; return fail(MGSA_ERR_NONFINITE, "z_j^T A z_j not finite");
    case mgsa::kDevTimeout: *info = -1; return fail(MGSA_ERR_TIMEOUT, "device-wide wait timed out");
    default: *info = -1; return fail(MGSA_ERR_CUDA, "unknown device status");
  }
}

mgsa_status mgsa_qr_host(mgsa_handle h, const int32_t* rowptr, const int32_t* col, const double* val,
                         int64_t nnz, const double* Z, int64_t m, int n, int64_t ldz, mgsa_variant v,
                         double* Q, int64_t ldq, double* R, int ldr, mgsa_stream_t s, int* info) {
  if (!h || !info) return fail(MGSA_ERR_INVALID, "NULL handle or info");
  if (!rowptr || !Z || !Q || !R || (nnz > 0 && (!col || !val))) return fail(MGSA_ERR_INVALID, "NULL host pointer");
  mgsa_status st = check_sizes(m, n, ldz, v, ldq, ldr);
  if (st != MGSA_OK) return st;
  if (nnz < 0 || nnz >= ((int64_t)1 << 31)) return fail(MGSA_ERR_INVALID, "nnz must be in [0, 2^31)");
  DeviceGuard g(h->device);
  if (!g.ok) return fail(MGSA_ERR_CUDA, "cannot select the device");
  // Device staging: rowptr | col | val | Z (ld m) | Q (ld m) | R (ld n), 256-byte aligned pieces.
  const size_t b_rp = (size_t)round_up(4 * (m + 1), 256), b_col = (size_t)round_up(4 * std::max<int64_t>(nnz, 1), 256);
  const size_t b_val = (size_t)round_up(8 * std::max<int64_t>(nnz, 1), 256), b_mat = (size_t)round_up(8 * m * n, 256);
  const size_t b_r = (size_t)round_up(8 * (int64_t)n * n, 256);
  const size_t need = b_rp + b_col + b_val + 2 * b_mat + b_r;
  if (need > h->io_bytes) {
    if (h->io) cudaFree(h->io);
    h->io = nullptr;
    h->io_bytes = 0;
    cudaError_t e = cudaMalloc(&h->io, need);
    if (e != cudaSuccess) return cuda_fail(e);
    h->io_bytes = need;
  }
  unsigned char* base = h->io;
  int32_t* d_rp = reinterpret_cast<int32_t*>(base);
  int32_t* d_col = reinterpret_cast<int32_t*>(base + b_rp);
  double* d_val = reinterpret_cast<double*>(base + b_rp + b_col);
  double* d_Z = reinterpret_cast<double*>(base + b_rp + b_col + b_val);
  double* d_Q = reinterpret_cast<double*>(base + b_rp + b_col + b_val + b_mat);
  double* d_R = reinterpret_cast<double*>(base + b_rp + b_col + b_val + 2 * b_mat);
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(s);
  cudaError_t e = cudaMemcpyAsync(d_rp, rowptr, 4 * (m + 1), cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess && nnz > 0) e = cudaMemcpyAsync(d_col, col, 4 * nnz, cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess && nnz > 0) e = cudaMemcpyAsync(d_val, val, 8 * nnz, cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(d_Z, 8 * m, Z, 8 * ldz, 8 * m, n, cudaMemcpyHostToDevice, cs);
  if (e != cudaSuccess) return cuda_fail(e);
  mgsa_csr A{m, nnz, d_rp, d_col, d_val};
  if ((st = mgsa_qr(h, &A, d_Z, m, n, m, v, d_Q, m, d_R, n, s)) != MGSA_OK) return st;
  e = cudaMemcpy2DAsync(Q, 8 * ldq, d_Q, 8 * m, 8 * m, n, cudaMemcpyDeviceToHost, cs);
  if (e == cudaSuccess) e = cudaMemcpy2DAsync(R, 8 * (size_t)ldr, d_R, 8 * n, 8 * n, n, cudaMemcpyDeviceToHost, cs);
  if (e != cudaSuccess) return cuda_fail(e);
  return mgsa_get_info(h, s, info);
}

}  // extern "C"
