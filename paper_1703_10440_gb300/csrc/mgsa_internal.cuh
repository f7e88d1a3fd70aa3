// Internal declarations shared by the CUDA translation units of libmgsa.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mgsa {

constexpr int kThreads = 512;             // threads per CTA of the single-instance kernel
constexpr int kWarps = kThreads / 32;
constexpr int kMaxChunk = 4096;           // rows whose pivots are staged in shared memory at once
constexpr int kMinRowsPerCta = 128;       // smallest row slab worth a CTA
constexpr int kMinRowsLongRows = 32;      // the same when rows are long (warp-per-row MVs)
constexpr unsigned long long kSpinLimitNs = 4000000000ull;  // 4 s bound on any device-wide wait

// Control block layout (int32 words, device memory, zeroed before each launch).
// kCtlBarCount counts CTA arrivals over the whole launch (barrier k completes at k * grid).
enum CtlWord { kCtlStatus = 0, kCtlColumn = 1, kCtlBarCount = 2, kCtlBarGen = 3, kCtlWords = 4 };

// Device status codes (equal to the public mgsa_status values).
enum DevStatus { kDevOk = 0, kDevBreakdown = 2, kDevNonfinite = 3, kDevTimeout = 6 };

enum Variant { kNaive = 0, kHA = 1, kHP = 2 };

struct SweepArgs {
  int64_t m;
  int n;
  const int32_t* rowptr;
  const int32_t* col;
  const double* val;
  const double* Z;
  int64_t ldz;
  double* Q;       // working z_j^{(i)} columns, then q_j
  int64_t ldq;
  double* R;
  int ldr;
  double* X;       // HP: m x n (x_j, then p_j); HA: x_i in column 0; naive: x_i, p_i in columns 0, 1
  int64_t ldx;
  double* part;    // (2(kg+n) + 1) * G partial sums: dots [parity][b][j] (two step-parity buffers), then norm [b]
  int* ctl;        // control block (CtlWord)
  int64_t rpc;     // rows per CTA, multiple of 32
  int chunk;       // rows per staged chunk, multiple of 32
  int mv_warp;     // 1: one warp per CSR row in the MVs / block product (long rows)
  int spmm_panel = 8;  // columns per pass of the block product X = A Z (4 or 8): selects the HP kernel
  // Successive orthogonalisation: kg given A-orthonormal columns Qg (with Pg =
  // their p_i) come first; the n columns of Z are columns kg .. kg+n-1 of the
  // virtual matrix and R is (kg+n) x n.  kg = 0 for a plain QR.
  int kg = 0;
  const double* Qg = nullptr;
  int64_t ldqg = 0;
  const double* Pg = nullptr;
  int64_t ldpg = 0;
  double* Pout = nullptr;  // optional p_j of the new columns (HA / naive; HP keeps them in X)
  int64_t ldpo = 0;
  // CGS only: q_j and p_j per CTA slab, block (j, b) = [q rows | p rows] of
  // rpc doubles each at qp + (j*G + b) * 2 * rpc; `stages` shared-memory
  // buffers of 2 * chunk doubles feed them to the update pass.
  double* qp = nullptr;
  int stages = 0;
  // Time slicing: this launch runs steps [step_begin, step_end) of the loop
  // (step_end < 0: to the end).  A slice that starts after step 0 reloads its
  // pivots and R row step_begin - 1 from global memory; one that ends early
  // sums its last R row in full.
  int step_begin = 0;
  int step_end = -1;
};

// Average row length from which a warp, not a thread, takes one CSR row.
constexpr int kWarpRowNnz = 32;

// Pivot rows of shared memory per chunk row: four in a resident slab (q and p
// of steps i-1 and i stay from one step to the next); in a staged slab q_{i-1},
// p_i and, for HP, p_{i-1}.  What shared memory a CTA leaves unused goes to
// its L1 cache, where the loads the fused pass keeps in flight land: on the
// 3D 128^3, n = 128 workload HP took 110.4 ms with 204 KB of shared memory
// per CTA against 98.7 ms with 138 KB; below that (HP 106 KB, HA 74 KB per
// CTA here) the time no longer changes.
__host__ __device__ constexpr int sweep_pivot_rows(bool resident, int variant) {
  return resident ? 4 : (variant == kHP ? 3 : 2);
}

// Shared memory bytes the single-instance kernel needs for n columns and a
// chunk, with piv_rows pivot rows per chunk row (4 covers every slab).
inline size_t sweep_smem_bytes(int n, int chunk, int piv_rows = 4) {
  const int kmax = (n + kWarps - 1) / kWarps + 2;
  return sizeof(double) * (size_t)(piv_rows * chunk + kWarps * kmax + 2 * n + kThreads + 1 + 8);
}

// One job of the batched kernel; same layout as mgsa_job in mgsa.h.
struct BatchJob {
  int64_t m;
  int32_t n;
  int32_t variant;
  const int32_t* rowptr;
  const int32_t* col;
  const double* val;
  const double* Z;
  int64_t ldz;
  double* Q;
  int64_t ldq;
  double* R;
  int64_t ldr;
  double* work;
};

constexpr int kBatchMaxN = 256;                 // largest n of a batched job
constexpr int kBatchInfoInvalid = -2147483647;  // info of a job rejected on the device

struct BatchArgs {
  const BatchJob* jobs;
  int count;
  int max_n;
  int* info;               // per job: 0, breakdown column, -column (non-finite), kBatchInfoInvalid
  unsigned int* queue;     // next job index per variant, 3 counters (zeroed before each launch)
  double* scratch;         // per-CTA partial sums
  int64_t scratch_stride;  // doubles per CTA, >= 2 * max_n + 1
  int row_mode = 0;        // 0: warp per row when nnz >= 32 m, 1: thread per row, 2: warp per row
  int spmm_panel = 8;      // as SweepArgs::spmm_panel, for every HP job
};

// Grouped launch: up to kGroupMax QRs side by side in one cooperative launch,
// each on a gang of CTAs of its own with its own device-wide barrier, each
// running a step range (a time slice) of its loop.
constexpr int kGroupMax = 64;
constexpr int kGroupCtlBytes = 256;  // member workspace: [ctl][partials][X columns]

struct GroupMember {
  BatchJob job;    // A, Z, Q, R, sizes; work = the member's workspace
  int first;       // steps [first, first + count) run in this launch
  int count;
  int G;           // CTAs of the gang
  int rpc;         // rows per CTA (multiple of 32)
  int chunk;       // rows per staged pivot chunk
  int mv_warp;     // one warp per CSR row in the MVs / block product (-1: decide from nnz = rowptr[m])
  int64_t part_doubles;  // per-CTA partial sums in the workspace
};

struct GroupArgs {
  int count;
  int spmm_panel;
  int offsets[kGroupMax + 1];  // first CTA of member k; offsets[count] = the grid
  GroupMember members[kGroupMax];
};

inline int64_t group_part_doubles(int n, int G) { return (int64_t)(2 * n + 1) * G; }

// Records the message mgsa_last_error returns on this thread (mgsa_api.cu).
void set_last_error(const char* why);

// Launch helpers (defined in mgsa_sweep.cu).
cudaError_t sweep_prepare(int device);  // sets shared-memory attributes once per device
cudaError_t sweep_max_ctas(int variant, size_t smem, int* max_ctas);
cudaError_t sweep_launch(int variant, const SweepArgs& a, int grid, size_t smem, cudaStream_t s);
cudaError_t group_max_ctas(int variant, size_t smem, int* max_ctas);
cudaError_t group_launch(int variant, const GroupArgs& ga, size_t smem, cudaStream_t s);

// One instance on one thread-block cluster of up to kMaxClusterCtas CTAs
// (non-portable sizes above 8 allowed where the GPU takes them).
constexpr int kMaxClusterCtas = 16;
cudaError_t cluster_prepare(int device);
cudaError_t cluster_max_size(int variant, size_t smem, int* max_size);
cudaError_t cluster_launch(int variant, const SweepArgs& a, int ctas, size_t smem, cudaStream_t s);

// Left-looking CGS kernels (mgsa_cgs.cu); variant = kNaive / kHA / kHP.
// X holds n columns (HP: x_j) or 2 (HA, naive: z_j, x_j); qp as in SweepArgs.
// cgs_smem_plan picks the number of pivot buffers that fit next to the rest.
constexpr int kCgsMaxStages = 8;
cudaError_t cgs_smem_plan(int variant, int n, int chunk, int* stages, size_t* smem);
cudaError_t cgs_prepare(int device);
cudaError_t cgs_max_ctas(int variant, size_t smem, int* max_ctas);
cudaError_t cgs_launch(int variant, const SweepArgs& a, int grid, size_t smem, cudaStream_t s);
cudaError_t batch_prepare(int device, size_t smem);
cudaError_t batch_max_ctas(size_t smem, int* max_ctas);
cudaError_t batch_launch(const BatchArgs& ba, int grid, size_t smem, cudaStream_t s);

}  // namespace mgsa
