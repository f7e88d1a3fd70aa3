// Single-instance A-inner-product MGS: one persistent cooperative kernel runs
// the whole right-looking loop (Algorithms 4, 7, 8 of Imakura & Yamamoto,
// arXiv 1703.10440) over row slabs owned by the CTAs.
//
// Every CTA owns rows [b*rpc, min(m, (b+1)*rpc)) of Z/Q and X for the whole
// kernel.  Step i of the loop is:
//
//   L   (i > 0) update column i with step i-1:  z_i -= r_{i-1,i} q_{i-1}
//               (HP also x_i -= r_{i-1,i} p_{i-1}); HP accumulates z_i^T x_i.
//   MV  (HA, naive) x_i = A z_i (the per-column MV of Algorithms 4/7),
//               accumulating z_i^T x_i.
//   D   r_ii = sqrt(sum of partials) (breakdown / non-finite check).
//   MV2 (naive) p_i = A q_i with q_i = z_i / r_ii gathered on the fly.
//   F   q_i = z_i / r_ii (stored), p_i = x_i / r_ii (eq. (tec1)); for every
//       j > i: apply step i-1's rank-1 updates z_j -= r_{i-1,j} q_{i-1}
//       (HP: x_j -= r_{i-1,j} p_{i-1}, eq. (tec2) one term at a time) and
//       accumulate r_ij = p_i^T z_j^{(i-1)}.
//
// so the updates of step i-1 and the dot products of step i share one pass
// over the remaining columns.  Division by r_ii is a multiplication by the
// reciprocal, formed once per step.
//
// Only r_{i,i+1} is needed before the next step's first barrier.  In a
// whole-GPU launch the other r_ij are summed once, spread over the CTAs, into
// R, and every CTA reloads them after that barrier; in a one-CTA (batched) or
// one-cluster launch every CTA sums them while that barrier is pending (split
// arrive / wait).  The per-CTA partials are double-buffered by step parity.
//
// On GB300 one warp-wide FP64 instruction holds the FP64 pipe for ~16 cycles,
// so every FP64 operation outside the fused pass is done once (not once per
// thread) or lane-per-column.  Reductions are deterministic: fixed trees and
// fixed orders that do not depend on timing; every CTA sums the G per-CTA
// partials in the same order.  Device-wide waits are bounded (kSpinLimitNs);
// on timeout the status word is set and every CTA returns.
#include "mgsa_device.cuh"

// Phase tracing (off unless compiled with -DMGSA_PHASE_TRACE): CTA 0 records
// %globaltimer at the phase boundaries of every step into g_mgsa_trace, which
// the traced build exports through mgsa_trace_fetch.  The product build
// contains neither.
#ifdef MGSA_PHASE_TRACE
__device__ unsigned long long g_mgsa_trace[4200][16];
extern "C" int mgsa_trace_fetch(unsigned long long* host) {
  return (int)cudaMemcpyFromSymbol(host, g_mgsa_trace, sizeof(g_mgsa_trace));
}
#define MGSA_TRACE(step, slot)                                            \
  do {                                                                    \
    if (blockIdx.x == 0 && threadIdx.x == 0) {                            \
      unsigned long long t_;                                              \
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_));              \
      g_mgsa_trace[(step)][(slot)] = t_;                                  \
    }                                                                     \
  } while (0)
#else
#define MGSA_TRACE(step, slot) ((void)0)
#endif

namespace mgsa {

namespace {

// r_{i,i+1}: the first entry of row i right of the diagonal (warp 0).  Column
// j of the virtual matrix is column j - kg of R.
__device__ void reduce_first(const double* part, int G, int nt, int i, double* s_rrow, double* R, int ldr, int kg,
                             bool write_r) {
  if (threadIdx.x < 32) {
    const double r = warp0_sum_ctas(part + (i + 1), nt, G);
    if (threadIdx.x == 0) {
      s_rrow[i + 1] = r;
      if (write_r) R[i + (int64_t)(i + 1 - kg) * ldr] = r;
    }
  }
  __syncthreads();
}

// Whole-GPU launches: row i of R is summed once, spread over the CTAs, instead
// of by every CTA.  Warp 0 sums r_{i,i+1} (needed at once by every CTA); the
// other warps of CTA b sum r_{i,j} for j = i + 2 + b + G t and store them in R.
// Each CTA reloads the row from R after the next step's first device-wide
// wait, which orders these stores before the loads.
__device__ void reduce_first_dist(const double* part, int G, int nt, int i, double* s_rrow, double* R, int ldr,
                                  int kg, int b) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (warp == 0) {
    const double r = warp_sum_ctas(part + (i + 1), nt, G, lane);
    if (lane == 0) {
      s_rrow[i + 1] = r;
      if (b == 0) R[i + (int64_t)(i + 1 - kg) * ldr] = r;
    }
  } else {
    for (int64_t j = i + 2 + b + (int64_t)G * (warp - 1); j < nt; j += (int64_t)G * (kWarps - 1)) {
      const double r = warp_sum_ctas(part + j, nt, G, lane);
      if (lane == 0) R[i + (j - kg) * ldr] = r;
    }
  }
  __syncthreads();
}

// Row i-1 of R, columns j > i (summed by reduce_first_dist at the end of step
// i-1), into s_rrow; warps 1.. load it while warp 0 forms the diagonal.
__device__ __forceinline__ void reload_row(const double* R, int ldr, int kg, int i, int nt, double* s_rrow) {
  if (threadIdx.x >= 32)
    for (int j = i + 1 + (int)threadIdx.x - 32; j < nt; j += kThreads - 32)
      s_rrow[j] = ld_cg(R + (i - 1) + (int64_t)(j - kg) * ldr);
}

constexpr int kTripRows = 8;                     // rows per lane per trip of the fused pass
constexpr int kMvRows = 4;                       // rows per thread in lockstep in the MVs of a staged slab (8, 16: slower)
constexpr int kMvEntries = 4;                    // entries per row loaded together in those MVs
// The first MV of a step (x_i = A z_i) gathers z_i through L1.  Safe: no CTA
// reads another CTA's rows of column i before this MV (the fused passes and
// the L update touch only a CTA's own rows, and slabs start on 256-byte
// boundaries, so no cache line holds rows of two slabs), so no stale line of
// those addresses can sit in this SM's L1.  Naive's second MV gathers q_i from
// the same addresses after they were rewritten and therefore reads L2.
constexpr bool kMvGatherL1 = true;
// Staged slabs of HA and naive: the rows of q_{i-1} that a chunk's fused pass
// reads are fetched into shared memory by one bulk copy (cp.async.bulk, this
// CTA's own rows of this GPU's memory), in flight while the threads form q_i
// and p_i; the rows of an odd tail are loaded by threads.  (3D 128^3, n = 128:
// HA 73.1 -> 72.3 ms.  HP, which also needs p_{i-1}, measured 99.1 -> 99.6 ms
// with two copies per chunk and keeps thread loads.)
template <int V>
constexpr bool kBulkStage = V != kHP;

// The fused pass over one chunk of rows [c0, c0 + crows) and the columns
// j = jbeg .. jbeg+ncols-1: apply step i-1's updates z_j -= r_{i-1,j} q_{i-1} (HP:
// x_j -= r_{i-1,j} p_{i-1}) and accumulate p_i^T z_j.  Work units are
// (column, 32-row block) pairs split into equal contiguous ranges, one per
// warp; each warp reduces each of its column pieces with a butterfly and the
// pieces are added in warp order into s_racc.  Pivots come from shared
// memory: s_qprev = q_{i-1}, s_pprev = p_{i-1}, s_pcur = p_i.
template <int V, bool kCross = false>
__device__ __forceinline__ void fused_pass(int i, int jbeg, int ncols, int kg, int64_t c0, int crows,
                                           const double* s_qprev, const double* s_pprev, const double* s_pcur,
                                           const double* s_rrow, double* __restrict__ Q, int64_t ldq,
                                           double* __restrict__ X, int64_t ldx, double* s_piece, int kmax,
                                           int* s_wfirst, int* s_wlast, double* s_racc) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nb = (crows + 31) >> 5;
  const int U = ncols * nb;  // <= 2047 * 128
  int u = (int)((int64_t)U * warp / kWarps);
  const int u1 = (int)((int64_t)U * (warp + 1) / kWarps);
  const int jfirst = u / nb;
  if (lane == 0) {
    s_wfirst[warp] = u < u1 ? jfirst : (1 << 30);
    s_wlast[warp] = u < u1 ? (u1 - 1) / nb : -1;
  }
  if (kCross) {
    // kCross: the warp's units are whole or partial columns in order; each column's
    // rows go in trips of kTripRows rows per lane.  Software-pipelined: as soon
    // as row q of a trip is done, the registers that held it are reloaded with
    // row q of the next trip -- of this column, or the first trip of the next
    // one -- so the next trip's loads are in flight while the rest of this
    // trip's FMAs run.  (The warps of a CTA move through the pass nearly in
    // lockstep, so loads issued only at the top of a trip, or of a column,
    // leave the FP64 pipe idle for a memory latency.)  Same operations, same
    // order as one trip at a time.  Trip counts and column changes are
    // warp-uniform; rows past the chunk are masked per lane.
    if (u < u1) {
      constexpr int kTrip = 32 * kTripRows;
      int jr = u / nb;
      int uend = (jr + 1) * nb < u1 ? (jr + 1) * nb : u1;
      int rb0 = (u - jr * nb) * 32;                       // first row of the column's range (warp-uniform)
      int ntrip = ((uend - jr * nb) * 32 - rb0 + kTrip - 1) / kTrip;
      int rend = (uend - jr * nb) * 32 < crows ? (uend - jr * nb) * 32 : crows;
      double rp = (i > 0) ? s_rrow[jbeg + jr] : 0.0;
      double* zc = Q + (int64_t)(jbeg + jr - kg) * ldq + c0;
      double* xc = (V == kHP) ? X + (int64_t)(jbeg + jr - kg) * ldx + c0 : X;
      double z[kTripRows], x[kTripRows];
  #pragma unroll
      for (int q = 0; q < kTripRows; ++q) {
        const int rr = rb0 + lane + 32 * q;
        z[q] = rr < rend ? zc[rr] : 0.0;
        x[q] = (V == kHP && i > 0 && rr < rend) ? xc[rr] : 0.0;
      }
      double acc0 = 0.0, acc1 = 0.0;
      for (int t = 0;;) {
        // The next trip: of this column, or the first of the next column.
        const bool col_end = t + 1 == ntrip;
        const bool more = !col_end || uend < u1;
        int rn0 = rb0 + (t + 1) * kTrip, rendn = rend;
        double* zcn = zc;
        double* xcn = xc;
        if (col_end && more) {
          const int jn = jr + 1;
          const int uendn = (jn + 1) * nb < u1 ? (jn + 1) * nb : u1;
          rn0 = 0;
          rendn = (uendn - jn * nb) * 32 < crows ? (uendn - jn * nb) * 32 : crows;
          zcn = Q + (int64_t)(jbeg + jn - kg) * ldq + c0;
          xcn = (V == kHP) ? X + (int64_t)(jbeg + jn - kg) * ldx + c0 : X;
        }
        const int r = rb0 + t * kTrip + lane;
  #pragma unroll
        for (int q = 0; q < kTripRows; ++q) {
          const int rr = r + 32 * q;
          if (rr < rend) {
            double zq = z[q];
            if (i > 0) {
              zq = fma(-rp, s_qprev[rr], zq);
              zc[rr] = zq;
              if (V == kHP) xc[rr] = fma(-rp, s_pprev[rr], x[q]);
            }
            if (q & 1) acc1 = fma(s_pcur[rr], zq, acc1);
            else acc0 = fma(s_pcur[rr], zq, acc0);
          }
          const int rq = rn0 + lane + 32 * q;
          const bool ld = more && rq < rendn;
          z[q] = ld ? zcn[rq] : 0.0;
          x[q] = (V == kHP && i > 0 && ld) ? xcn[rq] : 0.0;
        }
        if (!col_end) {
          ++t;
          continue;
        }
        const double acc = warp_sum(acc0 + acc1);
        if (lane == 0) s_piece[warp * kmax + (jr - jfirst)] = acc;
        if (!more) break;
        acc0 = acc1 = 0.0;
        ++jr;
        u = uend;
        uend = (jr + 1) * nb < u1 ? (jr + 1) * nb : u1;
        rb0 = 0;
        ntrip = ((uend - jr * nb) * 32 + kTrip - 1) / kTrip;
        rend = rendn;
        rp = (i > 0) ? s_rrow[jbeg + jr] : 0.0;
        zc = zcn;
        xc = xcn;
        t = 0;
      }
    }
  } else {
    while (u < u1) {
      const int jr = u / nb;
      const int j = jbeg + jr;  // column of the virtual matrix; column j - kg of Q / X
      const int uend = (jr + 1) * nb < u1 ? (jr + 1) * nb : u1;
      const double rp = (i > 0) ? s_rrow[j] : 0.0;
      double* zc = Q + (int64_t)(j - kg) * ldq + c0;
      double* xc = (V == kHP) ? X + (int64_t)(j - kg) * ldx + c0 : X;
      double acc0 = 0.0, acc1 = 0.0;
      const int rbeg = (u - jr * nb) * 32 + lane;
      int rend = (uend - jr * nb) * 32;
      if (rend > crows) rend = crows;
      // kTripRows rows per lane per trip.  Software-pipelined: as soon as row q
      // of a trip is done, the register that held it is reloaded with row q of
      // the next trip, so the next trip's loads are in flight while the rest of
      // this trip's FMAs run (the warps of a CTA move through the pass nearly in
      // lockstep, so loads issued only at the top of a trip would leave the
      // FP64 pipe idle for a memory latency per trip).  Same operations, same
      // order as one trip at a time.
      double z[kTripRows], x[kTripRows];
  #pragma unroll
      for (int q = 0; q < kTripRows; ++q) {
        const int rr = rbeg + 32 * q;
        z[q] = rr < rend ? zc[rr] : 0.0;
        x[q] = (V == kHP && i > 0 && rr < rend) ? xc[rr] : 0.0;
      }
      for (int r = rbeg; r < rend; r += 32 * kTripRows) {
        const int rn = r + 32 * kTripRows;  // next trip
  #pragma unroll
        for (int q = 0; q < kTripRows; ++q) {
          const int rr = r + 32 * q;
          if (rr < rend) {
            double zq = z[q];
            if (i > 0) {
              zq = fma(-rp, s_qprev[rr], zq);
              zc[rr] = zq;
              if (V == kHP) xc[rr] = fma(-rp, s_pprev[rr], x[q]);
            }
            if (q & 1) acc1 = fma(s_pcur[rr], zq, acc1);
            else acc0 = fma(s_pcur[rr], zq, acc0);
          }
          const int rq = rn + 32 * q;
          z[q] = rq < rend ? zc[rq] : 0.0;
          x[q] = (V == kHP && i > 0 && rq < rend) ? xc[rq] : 0.0;
        }
      }
      const double acc = warp_sum(acc0 + acc1);
      if (lane == 0) s_piece[warp * kmax + (jr - jfirst)] = acc;
      u = uend;
    }
  }
  __syncthreads();
  MGSA_TRACE(i, 5);
  // Combine the warp pieces of each column in warp order.
  for (int jr = threadIdx.x; jr < ncols; jr += kThreads) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w)
      if (jr >= s_wfirst[w] && jr <= s_wlast[w]) t += s_piece[w * kmax + (jr - s_wfirst[w])];
    s_racc[jr] += t;
  }
  __syncthreads();
}

// The whole right-looking loop for one instance, run by G CTAs (CTA b owns
// rows [b*rpc, (b+1)*rpc)).  Returns 0 or body_result(status, column).
// kSliced: the launch may be one time slice of the loop (steps [step_begin,
// step_end)); otherwise the whole loop, and none of the slicing code exists.
template <int V, bool kBatch, int kPanel, bool kSliced, bool kCluster = false>
__device__ int sweep_body(const SweepArgs& a, const int G, const int b, double* smem, int* s_wfirst, int* s_wlast,
                          int* s_flags) {
  // Row sums of R spread over the CTAs (whole-GPU launches), or summed by
  // every CTA (one CTA or one cluster per instance).
  constexpr bool kDist = !kBatch && !kCluster;
  const int n = a.n;    // columns of Z
  const int kg = a.kg;  // given columns before them (successive orthogonalisation)
  const int nt = kg + n;
  const int chunk = a.chunk;
  const int kmax = (nt + kWarps - 1) / kWarps + 2;
  // Resident mode: every slab is one chunk, so a CTA keeps q_{i-1}, p_{i-1}
  // in shared memory from one step to the next and its rows of z_i, x_i in
  // registers between the diagonal and the fused pass.
  const bool resident = a.rpc <= chunk;
  double* s_piv = smem;                                             // pivot rows (sweep_pivot_rows x chunk)
  double* s_piece = s_piv + sweep_pivot_rows(resident, V) * chunk;  // kWarps x kmax warp pieces
  double* s_racc = s_piece + kWarps * kmax;  // CTA partials of the current row (relative column)
  double* s_rrow = s_racc + nt;              // r_{i-1, j} during step i, then r_{i, j}
  double* s_buf = s_rrow + nt;               // kThreads + 1 reduction scratch
  double* s_scal = s_buf + kThreads + 1;     // r_ii, 1/r_ii, status

  const int tid = threadIdx.x;
  const int64_t m = a.m;
  const int64_t k0 = (int64_t)b * a.rpc;
  const int64_t k1 = (k0 + a.rpc < m) ? k0 + a.rpc : m;
  const int crows_all = (int)(k1 - k0);
  const int32_t* __restrict__ rowptr = a.rowptr;
  const int32_t* __restrict__ colidx = a.col;
  const double* __restrict__ val = a.val;
  const double* __restrict__ Z = a.Z;
  double* __restrict__ Q = a.Q;
  double* __restrict__ X = a.X;
  double* __restrict__ R = a.R;
  const int64_t ldz = a.ldz, ldq = a.ldq, ldx = a.ldx;
  const int ldr = a.ldr;
  // part: two buffers (step parity) of G x nt dot partials, then G norm partials.
  double* part_norm = a.part + 2 * (int64_t)nt * G;
  // One CTA per instance (batched): the CTA's own partials are the sums, so
  // z_i^T x_i and row i of R pass through registers and shared memory, not
  // through the scratch partials in L2.  (With one partial, the sums over
  // CTAs add only zeros: the same values.)
  double norm_local = 0.0;
  // Column j >= kg of the virtual matrix lives in column j - kg of Q and X, and
  // of R; the pivots of the given steps i < kg come from Qg and Pg.
  auto zcol = [&](int j) { return Q + (int64_t)(j - kg) * ldq; };
  auto xcol = [&](int j) { return X + (int64_t)(j - kg) * ldx; };
  auto qsrc = [&](int i) -> const double* { return i < kg ? a.Qg + (int64_t)i * a.ldqg : zcol(i); };
  auto psrc = [&](int i) -> const double* { return i < kg ? a.Pg + (int64_t)i * a.ldpg : xcol(i); };
  unsigned int gen = 0;
  // The mbarrier of the bulk-staged pivot rows (staged slabs only).
  __shared__ __align__(8) uint64_t s_bulk_bar_store;
  __shared__ int s_bulk_abort_store;
  uint64_t* s_bulk_bar = &s_bulk_bar_store;
  volatile int* s_bulk_abort = &s_bulk_abort_store;
  uint32_t bulk_phase = 0;
  if (kBulkStage<V> && !resident && tid == 0) {
    mbar_init(s_bulk_bar, 1);
    *s_bulk_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // Steps [i0, i1) run in this launch (time slicing; the whole loop by default).
  const int i0 = kSliced ? a.step_begin : 0;
  const int i1 = (!kSliced || a.step_end < 0 || a.step_end > nt) ? nt : a.step_end;

  MGSA_TRACE(4100, 0);
  if (!kSliced || i0 == 0) {
  // ---- Phase 0: R = 0; Q = Z on own rows; HP: X = A Z (one block product,
  // Algorithm 8 first line) and, outside resident mode, the partial z_1^T x_1. ----
  if (b == 0) {
    for (int64_t t = tid; t < (int64_t)nt * n; t += kThreads) R[(t % nt) + (t / nt) * ldr] = 0.0;
  }
  if (V == kHP) {
    const double s0 = spmm_slab_panel<kPanel>(rowptr, colidx, val, Z, ldz, X, ldx, Q, ldq, k0, k1, n, a.mv_warp != 0);
    if (!resident) {
      const double t = block_sum(s0, s_buf);
      norm_local = t;
      if (!kBatch && tid == 0) part_norm[b] = t;
    }
  } else {
    for (int j = 0; j < n; ++j)
      for (int64_t k = k0 + tid; k < k1; k += kThreads) Q[k + (int64_t)j * ldq] = __ldg(Z + k + (int64_t)j * ldz);
  }
  } else {
    // ---- A later slice: stop if an earlier one failed (the status word
    // survives between slices; no CTA writes it before the first wait, so
    // every CTA reads the same value).  Otherwise reload what the previous
    // slice left: R row i0-1 (summed in full at its end) and, in resident
    // mode, the pivots q_{i0-1} (Q) and p_{i0-1} (HP: X). ----
    if (ld_relaxed_i32(&a.ctl[kCtlStatus]) != 0) return 0;
    for (int j = i0 + tid; j < nt; j += kThreads) s_rrow[j] = ld_cg(R + (i0 - 1) + (int64_t)(j - kg) * ldr);
    if (resident) {
      double* sq = s_piv + 2 * ((i0 - 1) & 1) * chunk;
      const double* qg = qsrc(i0 - 1) + k0;
      const double* pg = psrc(i0 - 1) + k0;
      const int nb32 = ((crows_all + 31) >> 5) * 32;
      for (int r = tid; r < nb32; r += kThreads) {
        sq[r] = r < crows_all ? ld_cg(qg + r) : 0.0;
        if (V == kHP) sq[chunk + r] = r < crows_all ? ld_cg(pg + r) : 0.0;
      }
    }
  }
  __syncthreads();
  MGSA_TRACE(4100, 1);

  for (int i = i0; i < i1; ++i) {
    MGSA_TRACE(i, 0);
    const int cur = i & 1, prev = cur ^ 1;
    const bool given = i < kg;  // pivot q_i, p_i given (successive orthogonalisation)
    double* zi = given ? nullptr : zcol(i);
    const double* part_prev = a.part + (int64_t)prev * nt * G;  // partials of row i-1
    double* part_cur = a.part + (int64_t)cur * nt * G;          // partials of row i
    // The rest of row i-1 is summed during this step's first wait, unless row
    // i-1 was a given step's or the last of the previous slice (summed in full
    // right away).
    const bool rest_prev = i > kg && (!kSliced || i > i0);
    // This thread's rows tid + t*kThreads of z_i and x_i (naive: p_i), resident mode only.
    double zr[kResRows], xr[kResRows];
    // ---------------- column i: r_ii = sqrt(z_i^T x_i) ----------------
    double inv = 0.0;
    if (!given) {
    if (V == kHP) {
      if (resident) {
        const double r = (i > 0) ? s_rrow[i] : 0.0;  // r_{i-1,i}
        const double* xi = xcol(i);
        const double* sq = s_piv + 2 * prev * chunk;
        const double* sp = sq + chunk;
#pragma unroll
        for (int t = 0; t < kResRows; ++t) {
          const int rr = tid + t * kThreads;
          zr[t] = rr < crows_all ? zi[k0 + rr] : 0.0;
          xr[t] = rr < crows_all ? xi[k0 + rr] : 0.0;
        }
        double sl = 0.0;
#pragma unroll
        for (int t = 0; t < kResRows; ++t) {
          const int rr = tid + t * kThreads;
          if (rr < crows_all) {
            if (i > 0) {
              zr[t] = fma(-r, sq[rr], zr[t]);
              xr[t] = fma(-r, sp[rr], xr[t]);
            }
            sl = fma(zr[t], xr[t], sl);
          }
        }
        sl = block_sum(sl, s_buf);
        norm_local = sl;
        if (!kBatch && tid == 0) part_norm[b] = sl;
      } else if (i > 0) {
        const double r = s_rrow[i];  // r_{i-1,i}
        double sl = 0.0;
        double* xi = xcol(i);
        const double* qp = qsrc(i - 1);
        const double* pp = psrc(i - 1);
        // Four rows per thread per trip, loads first (rows stay in ascending order).
        for (int64_t k = k0 + tid; k < k1; k += 4 * kThreads) {
          double zz[4], xx[4], qq[4], pv[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int64_t kk = k + q * kThreads;
            const bool ok = kk < k1;
            zz[q] = ok ? zi[kk] : 0.0;
            xx[q] = ok ? xi[kk] : 0.0;
            qq[q] = ok ? qp[kk] : 0.0;
            pv[q] = ok ? pp[kk] : 0.0;
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int64_t kk = k + q * kThreads;
            if (kk < k1) {
              const double z = fma(-r, qq[q], zz[q]);
              const double x = fma(-r, pv[q], xx[q]);
              zi[kk] = z;
              xi[kk] = x;
              sl = fma(z, x, sl);
            }
          }
        }
        sl = block_sum(sl, s_buf);
        norm_local = sl;
        if (!kBatch && tid == 0) part_norm[b] = sl;
      }
      MGSA_TRACE(i, 1);
      sync_arrive<kBatch, kCluster>(a.ctl, gen, s_flags);
      if (!kDist && !kBatch && rest_prev)  // r_{i-1,j}, j > i
        reduce_range(part_prev, G, nt, i + 1, nt, s_rrow, s_buf, b == 0 ? R + (i - 1) : nullptr, ldr, kg);
      if (!sync_wait<kBatch, kCluster>(a.ctl, gen, (unsigned)G, s_flags)) return body_result(kDevTimeout, 0);
    } else {
      const double* zsrc;  // column i of the working Z, complete on every row
      if (i > 0) {
        const double r = s_rrow[i];
        const double* qp = qsrc(i - 1);
        if (resident) {
          const double* sq = s_piv + 2 * prev * chunk;
#pragma unroll
          for (int t = 0; t < kResRows; ++t) {
            const int rr = tid + t * kThreads;
            zr[t] = rr < crows_all ? zi[k0 + rr] : 0.0;
          }
#pragma unroll
          for (int t = 0; t < kResRows; ++t) {
            const int rr = tid + t * kThreads;
            if (rr < crows_all) {
              zr[t] = fma(-r, sq[rr], zr[t]);
              zi[k0 + rr] = zr[t];
            }
          }
        } else {
          for (int64_t k = k0 + tid; k < k1; k += 4 * kThreads) {
            double zz[4], qq[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int64_t kk = k + q * kThreads;
              zz[q] = kk < k1 ? zi[kk] : 0.0;
              qq[q] = kk < k1 ? qp[kk] : 0.0;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int64_t kk = k + q * kThreads;
              if (kk < k1) zi[kk] = fma(-r, qq[q], zz[q]);
            }
          }
        }
        MGSA_TRACE(i, 10);
        sync_arrive<kBatch, kCluster>(a.ctl, gen, s_flags);
        if (!kDist && !kBatch && rest_prev)
          reduce_range(part_prev, G, nt, i + 1, nt, s_rrow, s_buf, b == 0 ? R + (i - 1) : nullptr, ldr, kg);
        MGSA_TRACE(i, 11);
        if (!sync_wait<kBatch, kCluster>(a.ctl, gen, (unsigned)G, s_flags)) return body_result(kDevTimeout, 0);
        MGSA_TRACE(i, 12);
        zsrc = zi;
      } else {
        zsrc = Z;  // column 0 of the input equals the working column 0
        if (resident) {
#pragma unroll
          for (int t = 0; t < kResRows; ++t) {
            const int rr = tid + t * kThreads;
            zr[t] = rr < crows_all ? __ldg(Z + k0 + rr) : 0.0;
          }
        }
      }
      // x_i = A z_i^{(i-1)}  (Algorithm 4/7: the per-column MV)
      double sl = 0.0;
      if (a.mv_warp) {
        // One warp per row.  Resident mode: the row sums pass through this
        // step's p slot of the pivot buffer (free until the pivots are
        // formed) to the threads that own the rows.
        const int lane = tid & 31, warp = tid >> 5;
        double* xtmp = s_piv + (2 * cur + 1) * chunk;
        for (int64_t k = k0 + warp; k < k1; k += kWarps) {
          const double x = csr_row_warp<kMvGatherL1>(rowptr, colidx, val, zsrc, 1.0, false, k);
          if (lane == 0) {
            if (resident) {
              xtmp[k - k0] = x;
            } else {
              X[k] = x;
              sl = fma(ld_cg(zsrc + k), x, sl);
            }
          }
        }
        if (resident) {
          __syncthreads();
#pragma unroll
          for (int t = 0; t < kResRows; ++t) {
            const int rr = tid + t * kThreads;
            xr[t] = rr < crows_all ? xtmp[rr] : 0.0;
            if (rr < crows_all) sl = fma(zr[t], xr[t], sl);
          }
        }
      } else if (kBatch && resident) {
        // One CTA owns every row of the instance (k0 = 0): z_i goes to shared
        // memory (this step's q slot, free until the pivots) and the MV
        // gathers from there.
        double* s_z = s_piv + 2 * cur * chunk;
#pragma unroll
        for (int t = 0; t < kResRows; ++t) {
          const int rr = tid + t * kThreads;
          if (rr < crows_all) s_z[rr] = zr[t];
        }
        __syncthreads();
        if (crows_all > 4 * kThreads) {
          csr_rows_sh<kResRows>(rowptr, colidx, val, s_z, tid, k1, xr);
        } else {
          double xv[4];
          csr_rows_sh<4>(rowptr, colidx, val, s_z, tid, k1, xv);
#pragma unroll
          for (int q = 0; q < 4; ++q) xr[q] = xv[q];
#pragma unroll
          for (int q = 4; q < kResRows; ++q) xr[q] = 0.0;
        }
#pragma unroll
        for (int t = 0; t < kResRows; ++t)
          if (tid + t * kThreads < crows_all) sl = fma(zr[t], xr[t], sl);
      } else if (resident) {
        // All of a thread's rows in one lockstep round (one chain of
        // dependent loads) when it has more than four.
        if (crows_all > 4 * kThreads) {
          csr_rows<kResRows, kMvGatherL1>(rowptr, colidx, val, zsrc, 1.0, false, k0 + tid, k1, xr);
        } else {
          double xv[4];
          csr_rows<4, kMvGatherL1>(rowptr, colidx, val, zsrc, 1.0, false, k0 + tid, k1, xv);
#pragma unroll
          for (int q = 0; q < 4; ++q) xr[q] = xv[q];
#pragma unroll
          for (int q = 4; q < kResRows; ++q) xr[q] = 0.0;
        }
#pragma unroll
        for (int t = 0; t < kResRows; ++t)
          if (tid + t * kThreads < crows_all) sl = fma(zr[t], xr[t], sl);
      } else {
        for (int64_t k = k0 + tid; k < k1; k += kMvRows * kThreads) {
          double xv[kMvRows], zk[kMvRows];
          csr_rows_e<kMvRows, kMvEntries, kMvGatherL1>(rowptr, colidx, val, zsrc, 1.0, false, k, k1, xv);
#pragma unroll
          for (int q = 0; q < kMvRows; ++q) {
            const int64_t kk = k + q * kThreads;
            zk[q] = kk < k1 ? ld_cg(zsrc + kk) : 0.0;
          }
#pragma unroll
          for (int q = 0; q < kMvRows; ++q) {
            const int64_t kk = k + q * kThreads;
            if (kk < k1) {
              X[kk] = xv[q];
              sl = fma(zk[q], xv[q], sl);
            }
          }
        }
      }
      sl = block_sum(sl, s_buf);
      norm_local = sl;
      if (!kBatch && tid == 0) part_norm[b] = sl;
      MGSA_TRACE(i, 1);
      if (!sync_all<kBatch, kCluster>(a.ctl, gen, (unsigned)G, s_flags)) return body_result(kDevTimeout, 0);
    }
    MGSA_TRACE(i, 2);
    if (kDist && rest_prev) reload_row(R, ldr, kg, i, nt, s_rrow);  // r_{i-1,j}, j > i
    if (kBatch) diagonal_of(norm_local, s_scal);
    else diagonal(part_norm, G, s_scal);
    MGSA_TRACE(i, 3);
    if (s_scal[2] != 0.0) return body_result((int)s_scal[2], i + 1 - kg);  // the same verdict in every CTA
    inv = s_scal[1];
    if (b == 0 && tid == 0) R[i + (int64_t)(i - kg) * ldr] = s_scal[0];

    if (V == kNaive && resident) {
      // q_i = z_i / r_ii on this CTA's rows, into Q (no CTA reads z_i after
      // the norm wait); after the next wait the second MV of Algorithm 4,
      // p_i = A q_i, gathers it, with no multiply per nonzero.
      // Batched (one CTA owns every row, k0 = 0): q_i also into this step's q
      // slot of shared memory (the value the pivots store there later), and
      // the MV gathers from there.
      double* s_q = s_piv + 2 * cur * chunk;
#pragma unroll
      for (int t = 0; t < kResRows; ++t) {
        const int rr = tid + t * kThreads;
        if (rr < crows_all) {
          zi[k0 + rr] = zr[t] * inv;
          if (kBatch && !a.mv_warp) s_q[rr] = zr[t] * inv;
        }
      }
      if (!sync_all<kBatch, kCluster>(a.ctl, gen, (unsigned)G, s_flags)) return body_result(kDevTimeout, 0);
      if (kBatch && !a.mv_warp) {
        if (crows_all > 4 * kThreads) {
          csr_rows_sh<kResRows>(rowptr, colidx, val, s_q, tid, k1, xr);
        } else {
          double pv[4];
          csr_rows_sh<4>(rowptr, colidx, val, s_q, tid, k1, pv);
#pragma unroll
          for (int q = 0; q < 4; ++q) xr[q] = pv[q];
#pragma unroll
          for (int q = 4; q < kResRows; ++q) xr[q] = 0.0;
        }
      } else if (a.mv_warp) {
        const int lane = tid & 31, warp = tid >> 5;
        double* ptmp = s_piv + (2 * cur + 1) * chunk;
        for (int64_t k = k0 + warp; k < k1; k += kWarps) {
          const double pk = csr_row_warp(rowptr, colidx, val, zi, 1.0, false, k);
          if (lane == 0) ptmp[k - k0] = pk;
        }
        __syncthreads();
#pragma unroll
        for (int t = 0; t < kResRows; ++t) {
          const int rr = tid + t * kThreads;
          xr[t] = rr < crows_all ? ptmp[rr] : 0.0;
        }
      } else if (crows_all > 4 * kThreads) {
        csr_rows<kResRows>(rowptr, colidx, val, zi, 1.0, false, k0 + tid, k1, xr);
      } else {
        double pv[4];
        csr_rows4(rowptr, colidx, val, zi, 1.0, false, k0 + tid, k1, pv);
#pragma unroll
        for (int q = 0; q < 4; ++q) xr[q] = pv[q];
#pragma unroll
        for (int q = 4; q < kResRows; ++q) xr[q] = 0.0;
      }
    } else if (V == kNaive) {
      // p_i = A q_i with q_i = z_i / r_ii formed on the fly (Algorithm 4's second MV).
      const double* zsrc = (i > 0) ? zi : Z;
      if (a.mv_warp) {
        for (int64_t k = k0 + (tid >> 5); k < k1; k += kWarps) {
          const double pk = csr_row_warp(rowptr, colidx, val, zsrc, inv, true, k);
          if ((tid & 31) == 0) X[k + ldx] = pk;
        }
      } else {
        for (int64_t k = k0 + tid; k < k1; k += kMvRows * kThreads) {
          double pv[kMvRows];
          csr_rows_e<kMvRows, kMvEntries>(rowptr, colidx, val, zsrc, inv, true, k, k1, pv);
#pragma unroll
          for (int q = 0; q < kMvRows; ++q) {
            const int64_t kk = k + q * kThreads;
            if (kk < k1) X[kk + ldx] = pv[q];
          }
        }
      }
      // Other CTAs still gather z_i; q_i may overwrite it only after this wait.
      if (!sync_all<kBatch, kCluster>(a.ctl, gen, (unsigned)G, s_flags)) return body_result(kDevTimeout, 0);
    }
    }  // !given

    // ---------------- fused pass ----------------
    const int jbeg = i + 1 > kg ? i + 1 : kg;  // first working column right of pivot i
    const int ncols = nt - jbeg;
    for (int jr = tid; jr < ncols; jr += kThreads) s_racc[jr] = 0.0;
    if (resident) {
      // q_i = z_i / r_ii and p_i (eq. (tec1); naive: A q_i) from registers into
      // global memory and into this step's half of the pivot buffer.
      double* sqc = s_piv + 2 * cur * chunk;
      double* spc = sqc + chunk;
      const int nb32 = ((crows_all + 31) >> 5) * 32;
#pragma unroll
      for (int t = 0; t < kResRows; ++t) {
        const int rr = tid + t * kThreads;
        if (rr < nb32) {
          double qv = 0.0, pv = 0.0;
          if (rr < crows_all) {
            if (given) {
              qv = a.Qg[k0 + rr + (int64_t)i * a.ldqg];
              pv = a.Pg[k0 + rr + (int64_t)i * a.ldpg];
            } else {
              qv = zr[t] * inv;
              if (V != kNaive) zi[k0 + rr] = qv;  // naive: stored before its second MV
              pv = (V == kNaive) ? xr[t] : xr[t] * inv;
              if (V == kHP) xcol(i)[k0 + rr] = pv;
              else if (a.Pout) a.Pout[k0 + rr + (int64_t)(i - kg) * a.ldpo] = pv;
            }
          }
          sqc[rr] = qv;
          spc[rr] = pv;
        }
      }
      __syncthreads();
      MGSA_TRACE(i, 4);
      if (ncols > 0) {
        const double* sqp = s_piv + 2 * prev * chunk;
        fused_pass<V, true>(i, jbeg, ncols, kg, k0, crows_all, sqp, sqp + chunk, spc, s_rrow, Q, ldq, X, ldx, s_piece, kmax,
                      s_wfirst, s_wlast, s_racc);
      }
    } else {
      double* s_qprev = s_piv;
      double* s_pprev = s_piv + chunk;  // HP only
      double* s_pcur = s_piv + (V == kHP ? 2 : 1) * chunk;
      const double* const qprev = i > 0 ? qsrc(i - 1) : Q;
      const double* const pprev = (V == kHP && i > 0) ? psrc(i - 1) : X;
      const double* const qgiv = given ? qsrc(i) : Q;
      const double* xsrc = given ? psrc(i) : ((V == kHP) ? xcol(i) : (V == kHA ? X : X + ldx));
      for (int64_t c0 = k0; c0 < k1; c0 += chunk) {
        const int crows = (int)((k1 - c0) < chunk ? (k1 - c0) : chunk);
        const int nb = (crows + 31) >> 5;
        // Rows [0, brows) of q_{i-1} / p_{i-1} come by bulk copy (16-byte
        // aligned sources, an even row count), the rest by the threads.
        int brows = 0;
        if (kBulkStage<V> && i > 0 && (reinterpret_cast<uintptr_t>(qprev + c0) & 15) == 0) brows = crows & ~1;
        if (brows > 0 && tid == 0) {
          const uint32_t bytes = (uint32_t)brows * 8u;
          mbar_arrive_expect_tx(s_bulk_bar, bytes);
          bulk_load(s_qprev, qprev + c0, bytes, s_bulk_bar);
        }
        // Stage the pivots: q_i, p_i are formed (and stored), q_{i-1}, p_{i-1}
        // loaded.  Four rows per thread per trip, loads first.
        for (int r0 = tid; r0 < nb * 32; r0 += 4 * kThreads) {
          double zv[4], xv[4], qv[4], pv[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int r = r0 + q * kThreads;
            const bool ok = r < crows;
            const int64_t k = c0 + r;
            zv[q] = ok ? (given ? qgiv[k] : zi[k]) : 0.0;
            xv[q] = ok ? xsrc[k] : 0.0;
            qv[q] = (ok && i > 0 && r >= brows) ? qprev[k] : 0.0;
            pv[q] = (ok && i > 0 && V == kHP && r >= brows) ? pprev[k] : 0.0;
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int r = r0 + q * kThreads;
            if (r < nb * 32) {
              double pc = 0.0;
              if (r < crows && given) {
                pc = xv[q];  // given p_i
              } else if (r < crows) {
                const int64_t k = c0 + r;
                zi[k] = zv[q] * inv;  // q_i = z_i / r_ii
                if (V == kNaive) {
                  pc = xv[q];  // p_i = A q_i from the second MV
                } else {
                  pc = xv[q] * inv;  // p_i = x_i / r_ii (eq. (tec1))
                  if (V == kHP) xcol(i)[k] = pc;
                }
                if (V != kHP && a.Pout) a.Pout[k + (int64_t)(i - kg) * a.ldpo] = pc;
              }
              s_pcur[r] = pc;
              if (r >= brows) {
                s_qprev[r] = qv[q];
                if (V == kHP) s_pprev[r] = pv[q];
              }
            }
          }
        }
        if (kBulkStage<V>) fence_proxy_async_global();  // q_i is read by a bulk copy in the next step
        if (brows > 0) {
          if (!mbar_wait(s_bulk_bar, bulk_phase, s_bulk_abort)) {
            set_status(a.ctl, kDevTimeout, -1);
            return body_result(kDevTimeout, 0);
          }
          bulk_phase ^= 1u;
        }
        __syncthreads();
        MGSA_TRACE(i, 4);
        if (ncols > 0)
          fused_pass<V>(i, jbeg, ncols, kg, c0, crows, s_qprev, s_pprev, s_pcur, s_rrow, Q, ldq, X, ldx, s_piece,
                        kmax, s_wfirst, s_wlast, s_racc);
      }
    }
    MGSA_TRACE(i, 6);
    if (ncols == 0) break;
    if (kBatch && !given) {
      // Row i of R is this CTA's partials: straight into s_rrow and R (the
      // pass, the last reader of row i-1 in s_rrow, is complete).
      for (int jr = tid; jr < ncols; jr += kThreads) {
        s_rrow[jbeg + jr] = s_racc[jr];
        R[i + (int64_t)(jbeg + jr - kg) * ldr] = s_racc[jr];
      }
      __syncthreads();
      continue;
    }
    for (int jr = tid; jr < ncols; jr += kThreads) part_cur[(int64_t)b * nt + (jbeg + jr)] = s_racc[jr];
    MGSA_TRACE(i, 7);
    if (!sync_all<kBatch, kCluster>(a.ctl, gen, (unsigned)G, s_flags)) return body_result(kDevTimeout, 0);
    MGSA_TRACE(i, 8);
    if (given) {
      reduce_range(part_cur, G, nt, jbeg, nt, s_rrow, s_buf, b == 0 ? R + i : nullptr, ldr, kg);  // all of row i
    } else if (kDist) {
      // r_{i,i+1} here, r_{i,j} (j > i + 1) spread over the CTAs into R; a
      // later slice reloads the row from R as the next step would.
      reduce_first_dist(part_cur, G, nt, i, s_rrow, R, ldr, kg, b);
    } else {
      reduce_first(part_cur, G, nt, i, s_rrow, R, ldr, kg, b == 0);  // r_{i,i+1}; the rest at the next wait
    }
    MGSA_TRACE(i, 9);
  }
  return 0;
}

// Single instance over the whole grid (cooperative launch).
// kPanel: columns per pass of the block product (HP; one instantiation per width).
template <int V, int kPanel, bool kSliced>
__global__ void __launch_bounds__(kThreads, 1) mgs_sweep_kernel(const SweepArgs a) {
  extern __shared__ __align__(16) double smem[];
  __shared__ int s_wfirst[kWarps], s_wlast[kWarps];
  __shared__ int s_flags[2];
  const int r = sweep_body<V, false, kPanel, kSliced>(a, gridDim.x, blockIdx.x, smem, s_wfirst, s_wlast, s_flags);
  // Breakdown verdicts are identical in every CTA; CTA 0 records them.  A
  // timeout was recorded by the CTA that saw it.
  if (r != 0 && (r >> 24) != kDevTimeout && blockIdx.x == 0 && threadIdx.x == 0) set_status(a.ctl, r >> 24, r & 0xFFFFFF);
}

// Several instances side by side in one cooperative launch (a grouped launch):
// member k owns CTAs [offsets[k], offsets[k+1]) -- its gang -- and runs steps
// [first, first + count) of its loop over them with the time-slice body, its
// device-wide barriers counting only its own G CTAs on its own control words.
// No CTA waits for another member's, so members of any sizes share the GPU.
// For the same G, rows per CTA and chunk a member computes what mgsa_qr_steps
// computes with that plan, bit for bit.
template <int V, int kPanel>
__global__ void __launch_bounds__(kThreads, 1) mgs_group_kernel(const __grid_constant__ GroupArgs ga) {
  extern __shared__ __align__(16) double smem[];
  __shared__ int s_wfirst[kWarps], s_wlast[kWarps];
  __shared__ int s_flags[2];
  int k = 0;
  while (k + 1 < ga.count && (int)blockIdx.x >= ga.offsets[k + 1]) ++k;
  const GroupMember& M = ga.members[k];
  const int b = (int)blockIdx.x - ga.offsets[k];
  unsigned char* work = reinterpret_cast<unsigned char*>(M.job.work);
  SweepArgs a;
  a.m = M.job.m;
  a.n = M.job.n;
  a.rowptr = M.job.rowptr;
  a.col = M.job.col;
  a.val = M.job.val;
  a.Z = M.job.Z;
  a.ldz = M.job.ldz;
  a.Q = M.job.Q;
  a.ldq = M.job.ldq;
  a.R = M.job.R;
  a.ldr = (int)M.job.ldr;
  a.ctl = reinterpret_cast<int*>(work);
  a.part = reinterpret_cast<double*>(work + kGroupCtlBytes);
  a.X = a.part + M.part_doubles;
  a.ldx = (M.job.m + 31) / 32 * 32;
  a.rpc = M.rpc;
  a.chunk = M.chunk;
  a.mv_warp = M.mv_warp >= 0 ? M.mv_warp : (int64_t)__ldg(M.job.rowptr + M.job.m) >= (int64_t)kWarpRowNnz * M.job.m;
  a.spmm_panel = kPanel;
  a.step_begin = M.first;
  a.step_end = M.first + M.count;
  const int r = sweep_body<V, false, kPanel, true>(a, M.G, b, smem, s_wfirst, s_wlast, s_flags);
  if (r != 0 && (r >> 24) != kDevTimeout && b == 0 && threadIdx.x == 0) set_status(a.ctl, r >> 24, r & 0xFFFFFF);
}

// Before a grouped launch: every member's barrier counter starts at zero, and
// a member's first slice clears its status word too.
__global__ void group_reset_kernel(const __grid_constant__ GroupArgs ga) {
  for (int k = threadIdx.x; k < ga.count; k += blockDim.x) {
    int* ctl = reinterpret_cast<int*>(ga.members[k].job.work);
    ctl[kCtlBarCount] = 0;
    ctl[kCtlBarGen] = 0;
    if (ga.members[k].first == 0) {
      ctl[kCtlStatus] = 0;
      ctl[kCtlColumn] = 0;
    }
  }
}

// Single instance on one thread-block cluster (the whole grid): the same loop
// with hardware cluster barriers instead of the device-wide ones.  For
// problems too small to keep the whole GPU busy, where the per-step barrier
// latency, not the arithmetic, sets the time.
template <int V, int kPanel>
__global__ void __launch_bounds__(kThreads, 1) mgs_cluster_kernel(const SweepArgs a) {
  extern __shared__ __align__(16) double smem[];
  __shared__ int s_wfirst[kWarps], s_wlast[kWarps];
  __shared__ int s_flags[2];
  const int r = sweep_body<V, false, kPanel, false, true>(a, gridDim.x, blockIdx.x, smem, s_wfirst, s_wlast, s_flags);
  if (r != 0 && blockIdx.x == 0 && threadIdx.x == 0) set_status(a.ctl, r >> 24, r & 0xFFFFFF);
}

// Many independent instances: every CTA takes the next job from the queue and
// runs the whole loop of that instance by itself (CTA-wide barriers only).
// One launch per variant: the launch for V takes the jobs of variant V (the
// HP launch also answers jobs whose variant is unknown).
template <int V, int kPanel>
__global__ void __launch_bounds__(kThreads, 1) mgs_batch_kernel(const BatchArgs ba) {
  extern __shared__ __align__(16) double smem[];
  __shared__ int s_wfirst[kWarps], s_wlast[kWarps];
  __shared__ int s_flags[2];
  __shared__ int s_job;
  double* part = ba.scratch + (int64_t)blockIdx.x * ba.scratch_stride;
  for (;;) {
    if (threadIdx.x == 0) s_job = (int)atomicAdd(ba.queue + V, 1u);
    __syncthreads();
    const int jb = s_job;
    __syncthreads();
    if (jb >= ba.count) break;
    const BatchJob& J = ba.jobs[jb];
    const int64_t m = J.m;
    const int n = J.n;
    const bool known = J.variant >= kNaive && J.variant <= kHP;
    if (J.variant != V && (known || V != kHP)) continue;  // another launch's job
    int result;
    if (!known || n < 1 || n > ba.max_n || m < n || m >= ((int64_t)1 << 31) || J.ldz < m || J.ldq < m ||
        J.ldr < n || !J.rowptr || !J.Z || !J.Q || !J.R || !J.work) {
      result = -1;
    } else {
      SweepArgs a;
      a.m = m;
      a.n = n;
      a.rowptr = J.rowptr;
      a.col = J.col;
      a.val = J.val;
      a.Z = J.Z;
      a.ldz = J.ldz;
      a.Q = J.Q;
      a.ldq = J.ldq;
      a.R = J.R;
      a.ldr = (int)J.ldr;
      a.X = J.work;
      a.ldx = (m + 31) / 32 * 32;
      a.part = part;
      a.ctl = nullptr;
      a.rpc = (m + 31) / 32 * 32;
      a.chunk = (int)(a.rpc < kMaxChunk ? a.rpc : kMaxChunk);
      a.mv_warp = ba.row_mode == 0 ? (int64_t)__ldg(J.rowptr + m) >= (int64_t)kWarpRowNnz * m : ba.row_mode == 2;
      result = sweep_body<V, true, kPanel, false>(a, 1, 0, smem, s_wfirst, s_wlast, s_flags);
    }
    if (threadIdx.x == 0) {
      int info = 0;
      if (result == -1) info = kBatchInfoInvalid;
      else if ((result >> 24) == kDevBreakdown) info = result & 0xFFFFFF;
      else if ((result >> 24) == kDevNonfinite) info = -(result & 0xFFFFFF);
      ba.info[jb] = info;
    }
    __syncthreads();
  }
}

}  // namespace

// The kernels: naive and HA have no block product; HP has one per panel
// width; each also as a time-slice instance.
template <bool kSliced>
static const void* sweep_fn_s(int variant, int panel) {
  switch (variant) {
    case kNaive: return reinterpret_cast<const void*>(mgs_sweep_kernel<kNaive, 8, kSliced>);
    case kHA: return reinterpret_cast<const void*>(mgs_sweep_kernel<kHA, 8, kSliced>);
    default:
      return panel == 4 ? reinterpret_cast<const void*>(mgs_sweep_kernel<kHP, 4, kSliced>)
                        : reinterpret_cast<const void*>(mgs_sweep_kernel<kHP, 8, kSliced>);
  }
}

static const void* sweep_fn(int variant, int panel = 8, bool sliced = false) {
  return sliced ? sweep_fn_s<true>(variant, panel) : sweep_fn_s<false>(variant, panel);
}

static const void* batch_fn(int variant, int panel = 8) {
  switch (variant) {
    case kNaive: return reinterpret_cast<const void*>(mgs_batch_kernel<kNaive, 8>);
    case kHA: return reinterpret_cast<const void*>(mgs_batch_kernel<kHA, 8>);
    default:
      return panel == 4 ? reinterpret_cast<const void*>(mgs_batch_kernel<kHP, 4>)
                        : reinterpret_cast<const void*>(mgs_batch_kernel<kHP, 8>);
  }
}

// Every kernel instance: (variant, panel width).
static const int kKernelInstances[4][2] = {{kNaive, 8}, {kHA, 8}, {kHP, 8}, {kHP, 4}};

static const void* group_fn(int variant, int panel = 8) {
  switch (variant) {
    case kNaive: return reinterpret_cast<const void*>(mgs_group_kernel<kNaive, 8>);
    case kHA: return reinterpret_cast<const void*>(mgs_group_kernel<kHA, 8>);
    default:
      return panel == 4 ? reinterpret_cast<const void*>(mgs_group_kernel<kHP, 4>)
                        : reinterpret_cast<const void*>(mgs_group_kernel<kHP, 8>);
  }
}

cudaError_t sweep_prepare(int device) {
  int optin = 0;
  cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  if (e != cudaSuccess) return e;
  for (const auto& k : kKernelInstances) {
    for (const void* fn : {sweep_fn(k[0], k[1], false), sweep_fn(k[0], k[1], true), group_fn(k[0], k[1])}) {
      cudaFuncAttributes fa;
      if ((e = cudaFuncGetAttributes(&fa, fn)) != cudaSuccess) return e;
      const int dyn = optin - (int)fa.sharedSizeBytes;  // static shared memory counts against the opt-in limit
      if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn)) != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

static const void* cluster_fn(int variant, int panel = 8) {
  switch (variant) {
    case kNaive: return reinterpret_cast<const void*>(mgs_cluster_kernel<kNaive, 8>);
    case kHA: return reinterpret_cast<const void*>(mgs_cluster_kernel<kHA, 8>);
    default:
      return panel == 4 ? reinterpret_cast<const void*>(mgs_cluster_kernel<kHP, 4>)
                        : reinterpret_cast<const void*>(mgs_cluster_kernel<kHP, 8>);
  }
}

cudaError_t cluster_prepare(int device) {
  int optin = 0;
  cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  if (e != cudaSuccess) return e;
  for (const auto& k : kKernelInstances) {
    const void* fn = cluster_fn(k[0], k[1]);
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, fn)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes)) !=
        cudaSuccess)
      return e;
    if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t cluster_max_size(int variant, size_t smem, int* max_size) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kMaxClusterCtas);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kMaxClusterCtas;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int size = 0;
  cudaError_t e = cudaOccupancyMaxPotentialClusterSize(&size, cluster_fn(variant), &cfg);
  if (e != cudaSuccess) return e;
  *max_size = size < kMaxClusterCtas ? size : kMaxClusterCtas;
  return cudaSuccess;
}

cudaError_t cluster_launch(int variant, const SweepArgs& a, int ctas, size_t smem, cudaStream_t s) {
  SweepArgs copy = a;
  void* args[] = {&copy};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ctas);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = ctas;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, cluster_fn(variant, a.spmm_panel), args);
}

cudaError_t sweep_max_ctas(int variant, size_t smem, int* max_ctas) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_fn(variant), kThreads, smem)) != cudaSuccess) return e;
  *max_ctas = sms * per_sm;
  return cudaSuccess;
}

cudaError_t batch_prepare(int device, size_t smem) {
  int optin = 0;
  cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  if (e != cudaSuccess) return e;
  for (const auto& k : kKernelInstances) {
    const void* fn = batch_fn(k[0], k[1]);
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, fn)) != cudaSuccess) return e;
    if (smem + fa.sharedSizeBytes > (size_t)optin) return cudaErrorInvalidValue;
    if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t batch_max_ctas(size_t smem, int* max_ctas) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_fn(kHP), kThreads, smem)) != cudaSuccess)
    return e;
  *max_ctas = sms * per_sm;
  return cudaSuccess;
}

cudaError_t batch_launch(const BatchArgs& ba, int grid, size_t smem, cudaStream_t s) {
  mgs_batch_kernel<kNaive, 8><<<grid, kThreads, smem, s>>>(ba);
  mgs_batch_kernel<kHA, 8><<<grid, kThreads, smem, s>>>(ba);
  if (ba.spmm_panel == 4) mgs_batch_kernel<kHP, 4><<<grid, kThreads, smem, s>>>(ba);
  else mgs_batch_kernel<kHP, 8><<<grid, kThreads, smem, s>>>(ba);
  return cudaGetLastError();
}

cudaError_t group_max_ctas(int variant, size_t smem, int* max_ctas) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, group_fn(variant), kThreads, smem)) != cudaSuccess)
    return e;
  *max_ctas = sms * per_sm;
  return cudaSuccess;
}

cudaError_t group_launch(int variant, const GroupArgs& ga, size_t smem, cudaStream_t s) {
  group_reset_kernel<<<1, 64, 0, s>>>(ga);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  void* args[] = {const_cast<GroupArgs*>(&ga)};
  return cudaLaunchCooperativeKernel(group_fn(variant, ga.spmm_panel), dim3(ga.offsets[ga.count]), dim3(kThreads),
                                     args, smem, s);
}

cudaError_t sweep_launch(int variant, const SweepArgs& a, int grid, size_t smem, cudaStream_t s) {
  SweepArgs copy = a;
  void* args[] = {&copy};
  const bool sliced = a.step_begin != 0 || a.step_end >= 0;
  return cudaLaunchCooperativeKernel(sweep_fn(variant, a.spmm_panel, sliced), dim3(grid), dim3(kThreads), args, smem,
                                     s);
}

}  // namespace mgsa
