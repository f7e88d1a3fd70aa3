// Classical Gram-Schmidt under the A-inner product -- CGS-naive, CGS-HA and
// CGS-HP (Section 2.3 of Imakura & Yamamoto, arXiv 1703.10440; recurrences in
// Section 3.3) -- as one persistent cooperative kernel, column by column
// (left-looking).
//
// CGS takes every coefficient of column j against the original column,
// r_ij = p_i^T z_j^{(0)} (i < j), so the whole column of coefficients is one
// GEMV-shaped product P^T z_j^{(0)} that needs nothing of column j but its
// input.  Column j of the loop:
//
//   U   z_j = z_j^{(0)} - sum_{i<j} r_ij q_i   (HP also x_j = x_j^{(0)} -
//       sum_{i<j} r_ij p_i, eq. (tec2)); the same pass over q_i, p_i forms the
//       CTA's partial products p_i^T z_{j+1}^{(0)} of the next column.
//   MV  (HA, naive) x_j = A z_j.
//   D   r_jj = sqrt(z_j^T x_j), breakdown check.
//   MV2 (naive) p_j = A q_j, q_j formed on the fly.
//   F   q_j = z_j / r_jj, p_j = x_j / r_jj (eq. (tec1)); p_j^T z_{j+1}^{(0)}.
//
// Device-wide waits per column: HP two (the norm after U; r_{j,j+1} after F),
// HA and naive three (the MV gathers z_j from other CTAs' rows).  Every CTA
// sums r_{j,j+1} after the last wait of column j; r_{i,j+1} (i < j) are summed
// once, spread over the CTAs (CTA b takes i = b + G t), off the critical path,
// stored in R and reloaded by every CTA after that wait.  CTA b owns rows
// [b*rpc, (b+1)*rpc) of every column; only the MV gathers and the partial
// sums cross CTAs.
//
// U streams every earlier pivot once per column.  F stores q_j, p_j of the
// CTA's rows as one contiguous block per (pivot, CTA), and U fetches each
// block with one bulk asynchronous copy (cp.async.bulk, completion counted on
// an mbarrier) into a ring of shared-memory buffers, several pivots ahead of
// the arithmetic, so the FP64 pipe -- not the load latency -- sets the pace.
// One thread issues the copies; each warp releases a buffer (second mbarrier)
// when it is done with it.  Every wait is bounded (kSpinLimitNs).
//
// Rows sit in registers (row tid + t*kThreads in slot t) during U and F when
// a CTA's slab is one chunk; otherwise U and F stream the slab chunk by chunk
// and keep z_j, x_j in memory in between.  Division by r_jj is a
// multiplication by its reciprocal.  Reductions use fixed trees and orders.
//
// Workspace X (leading dimension ldx): HP: column j holds x_j^{(0)} = (A Z)_j
// (staged mode: then x_j); HA/naive: column 0 the copy of z_j that the MVs
// gather, column 1 x_j (staged mode).
#include "mgsa_device.cuh"

// Phase tracing (off unless compiled with -DMGSA_PHASE_TRACE): CTA 0 records
// %globaltimer at the phase boundaries of every column into g_cgs_trace,
// exported by the traced build through mgsa_cgs_trace_fetch.
#ifdef MGSA_PHASE_TRACE
__device__ unsigned long long g_cgs_trace[4200][12];
extern "C" int mgsa_cgs_trace_fetch(unsigned long long* host) {
  return (int)cudaMemcpyFromSymbol(host, g_cgs_trace, sizeof(g_cgs_trace));
}
#define CGS_TRACE(col, slot)                                              \
  do {                                                                    \
    if (blockIdx.x == 0 && threadIdx.x == 0) {                            \
      unsigned long long t_;                                              \
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_));              \
      g_cgs_trace[(col)][(slot)] = t_;                                    \
    }                                                                     \
  } while (0)
#else
#define CGS_TRACE(col, slot) ((void)0)
#endif

namespace mgsa {

namespace {

constexpr int kGroup = 8;       // pivots whose dot partials one thread carries at once
constexpr int kPieceCols = 64;  // pivots per flush of the per-warp partial sums

// Sums of v[0..7] over the 32 lanes of a warp: three halving exchanges (lane
// l keeps the entries selected by its bits 4, 3, 2) leave lane l with the sum
// of v[(l >> 2) & 7] over 8 lanes; two butterflies complete it.  Lanes with
// (l & 3) == 0 then hold the full sum of v[(l >> 2) & 7].  A fixed tree.
__device__ __forceinline__ double warp_sum8(double v[kGroup]) {
  const int lane = threadIdx.x & 31;
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double send = b4 ? v[k] : v[k + 4];
    const double keep = b4 ? v[k + 4] : v[k];
    v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const double send = b3 ? v[k] : v[k + 2];
    const double keep = b3 ? v[k + 2] : v[k];
    v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  const double send = b2 ? v[0] : v[1];
  const double keep = b2 ? v[1] : v[0];
  double t = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  t += __shfl_xor_sync(0xffffffffu, t, 2);
  t += __shfl_xor_sync(0xffffffffu, t, 1);
  return t;
}

// Ring of pivot buffers.  Copy number s (counted over the whole kernel) goes
// to buffer s % S; its use u = s / S completes phase u of full[s % S] and,
// once all warps are done with it, phase u of empty[s % S].
struct PivotRing {
  uint64_t* full;
  uint64_t* empty;
  double* buf;      // S buffers of 2 * chunk doubles: [q rows | p rows]
  int S;
  int chunk;
  unsigned next;    // next copy to consume (same value in every thread)
  unsigned issued;  // next copy to issue (meaningful in thread 0)
  volatile int* abort;  // raised by the first wait that gives up
};

// After a failed wait: thread 0 waits, for at most kSpinLimitNs in all, for
// the copies it issued that nobody has waited for, so that none is still
// writing this CTA's shared memory when the CTA leaves.
__device__ void ring_drain(PivotRing& r, unsigned from) {
  const unsigned long long t0 = global_timer_ns();
  for (unsigned s = from; s < r.issued; ++s) {
    const int slot = (int)(s % (unsigned)r.S);
    while (!mbar_try_wait(&r.full[slot], (s / (unsigned)r.S) & 1u))
      if (global_timer_ns() - t0 > kSpinLimitNs) return;
  }
}

// Thread 0: copy `rows` doubles of q_i (from qsrc) and of p_i (from psrc)
// into the next buffer, once every warp has released that buffer's previous
// use.  False if that wait timed out (nothing is issued then).
__device__ __forceinline__ bool ring_issue(PivotRing& r, const double* qsrc, const double* psrc, int rows) {
  const unsigned s = r.issued;
  const int slot = (int)(s % (unsigned)r.S);
  const unsigned use = s / (unsigned)r.S;
  if (use > 0 && !mbar_wait(&r.empty[slot], (use - 1) & 1u, r.abort)) return false;
  r.issued = s + 1;
  const uint32_t bytes = (uint32_t)rows * (uint32_t)sizeof(double);
  double* dst = r.buf + (int64_t)slot * 2 * r.chunk;
  mbar_arrive_expect_tx(&r.full[slot], 2 * bytes);
  bulk_load(dst, qsrc, bytes, &r.full[slot]);
  bulk_load(dst + r.chunk, psrc, bytes, &r.full[slot]);
  return true;
}

// The U pass over one chunk of rows [c0, c0 + crows) of CTA b, slot t of
// this thread being row tid + t*kThreads of the chunk: for i = 0 .. j-1 in
// order,
//   z -= r_ij q_i,  (HP) x -= r_ij p_i,  d_i += p_i . z1
// with z1 the rows of z_{j+1}^{(0)}; q_i, p_i arrive through the ring from
// block (i, b) of qp (rows padded to 32, blk = rpc doubles per half).  When
// `dots` is set, the chunk's d_i (slots in order within a thread, a fixed tree
// within a warp, warps in order) are stored to dots[i] (accumulate: added).
// Slots beyond the chunk are skipped warp by warp.  Returns false if a wait
// timed out (in any thread of the CTA).
template <int V>
__device__ bool update_pass(int j, int crows, const double* qp_cta, int64_t cta_stride, int64_t blk, int64_t off,
                            const double* s_r, PivotRing& ring, double zr[kResRows], double xr[kResRows],
                            const double z1r[kResRows], double* dots, bool accumulate, double* s_piece) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int rows = (crows + 31) & ~31;
  const int S = ring.S;
  bool ok = true;
  // pivot i's rows: q at qp_cta + i * cta_stride + off, p blk doubles later
  if (tid == 0) {
    const int pre = j < S ? j : S;
    for (int i = 0; i < pre && ok; ++i) {
      const double* q = qp_cta + (int64_t)i * cta_stride + off;
      ok = ring_issue(ring, q, q + blk, rows);
    }
  }
  const unsigned base = ring.next;
  for (int ib = 0; ib < j; ib += kPieceCols) {
    const int iend = (j - ib) < kPieceCols ? j : ib + kPieceCols;
    for (int i0 = ib; i0 < iend; i0 += kGroup) {
      double acc[kGroup];
#pragma unroll
      for (int g = 0; g < kGroup; ++g) acc[g] = 0.0;
#pragma unroll
      for (int g = 0; g < kGroup; ++g) {
        const int i = i0 + g;
        if (i < iend) {
          const unsigned s = base + (unsigned)i;
          const int slot = (int)(s % (unsigned)S);
          if (ok && !mbar_wait(&ring.full[slot], (s / (unsigned)S) & 1u, ring.abort)) ok = false;
          const double* sq = ring.buf + (int64_t)slot * 2 * ring.chunk;
          const double* sp = sq + ring.chunk;
          const double r = s_r[i];
#pragma unroll
          for (int t = 0; t < kResRows; ++t) {
            if (t * kThreads + (warp << 5) < crows) {
              const int rr = tid + t * kThreads;
              const bool in = rr < crows;
              const double qv = in ? sq[rr] : 0.0;
              const double pv = in ? sp[rr] : 0.0;
              zr[t] = fma(-r, qv, zr[t]);
              if (V == kHP) xr[t] = fma(-r, pv, xr[t]);
              acc[g] = fma(pv, z1r[t], acc[g]);
            }
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(&ring.empty[slot]);
          // refill the buffer of pivot i-1 (released by every warp by now, or soon)
          if (tid == 0 && ok && i >= 1 && i - 1 + S < j) {
            const double* q = qp_cta + (int64_t)(i - 1 + S) * cta_stride + off;
            ok = ring_issue(ring, q, q + blk, rows);
          }
        }
      }
      if (dots) {
        const double w = warp_sum8(acc);
        if ((lane & 3) == 0) s_piece[warp * kPieceCols + (i0 - ib) + ((lane >> 2) & 7)] = w;
      }
    }
    if (dots) {
      __syncthreads();
      for (int t = tid; t < iend - ib; t += kThreads) {
        double sum = s_piece[t];
#pragma unroll
        for (int w = 1; w < kWarps; ++w) sum += s_piece[w * kPieceCols + t];
        dots[ib + t] = accumulate ? dots[ib + t] + sum : sum;
      }
      __syncthreads();
    }
  }
  ring.next = base + (unsigned)j;
  if (__syncthreads_or(!ok)) {
    if (tid == 0) ring_drain(ring, base);
    return false;
  }
  return true;
}

// Loads rows [c0, c0 + crows) of a column into the slots of this thread.
__device__ __forceinline__ void load_slots(const double* col, int64_t c0, int crows, double v[kResRows]) {
#pragma unroll
  for (int t = 0; t < kResRows; ++t) {
    const int rr = threadIdx.x + t * kThreads;
    v[t] = (col && rr < crows) ? ld_cg(col + c0 + rr) : 0.0;
  }
}

// x = A src on the rows [k0, k1) of this CTA.  Resident (k1 - k0 <= chunk):
// into the slots xr (long rows pass through s_xtmp); staged: into xout[k].
// Returns this thread's share of sum_k z[k] x[k] (z = the slots zr when
// resident, src itself when staged) if want_dot.
__device__ double mv_rows(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                          const double* __restrict__ val, const double* src, double scale, bool scale_src,
                          int64_t k0, int64_t k1, bool resident, bool warp_rows, double xr[kResRows],
                          const double zr[kResRows], double* xout, double* s_xtmp, bool want_dot) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int crows = (int)(k1 - k0);
  double sl = 0.0;
  if (warp_rows) {
    for (int64_t k = k0 + warp; k < k1; k += kWarps) {
      const double x = csr_row_warp(rowptr, colidx, val, src, scale, scale_src, k);
      if (lane == 0) {
        if (resident) {
          s_xtmp[k - k0] = x;
        } else {
          xout[k] = x;
          if (want_dot) sl = fma(ld_cg(src + k), x, sl);
        }
      }
    }
    if (resident) {
      __syncthreads();
#pragma unroll
      for (int t = 0; t < kResRows; ++t) {
        const int rr = tid + t * kThreads;
        xr[t] = rr < crows ? s_xtmp[rr] : 0.0;
        if (want_dot && rr < crows) sl = fma(zr[t], xr[t], sl);
      }
      __syncthreads();  // s_xtmp is reused by the next MV
    }
  } else if (resident) {
#pragma unroll
    for (int h = 0; h < kResRows / 4; ++h) {
      double xv[4] = {0.0, 0.0, 0.0, 0.0};
      if (h * 4 * kThreads < crows)
        csr_rows4(rowptr, colidx, val, src, scale, scale_src, k0 + tid + (int64_t)h * 4 * kThreads, k1, xv);
#pragma unroll
      for (int q = 0; q < 4; ++q) xr[4 * h + q] = xv[q];
    }
    if (want_dot) {
#pragma unroll
      for (int t = 0; t < kResRows; ++t)
        if (tid + t * kThreads < crows) sl = fma(zr[t], xr[t], sl);
    }
  } else {
    for (int64_t k = k0 + tid; k < k1; k += 4 * kThreads) {
      double xv[4], zk[4];
      csr_rows4(rowptr, colidx, val, src, scale, scale_src, k, k1, xv);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int64_t kk = k + q * kThreads;
        zk[q] = (want_dot && kk < k1) ? ld_cg(src + kk) : 0.0;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int64_t kk = k + q * kThreads;
        if (kk < k1) {
          xout[kk] = xv[q];
          if (want_dot) sl = fma(zk[q], xv[q], sl);
        }
      }
    }
  }
  return sl;
}

// r_{i,j+1}, i < j, summed once over the CTAs: warps 1.. of CTA b sum the
// entries i = b + G t (the partials of every CTA are complete) and store them
// in column j+1 of R; every CTA reloads that column after the column's last
// device-wide wait.  Warp 0 is left free for the diagonal.
__device__ __forceinline__ void sum_assigned(const double* part, int G, int n, int j, double* R, int ldr, int b) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (warp == 0) return;
  for (int64_t i = b + (int64_t)G * (warp - 1); i < j; i += (int64_t)G * (kWarps - 1)) {
    const double r = warp_sum_ctas(part + i, n, G, lane);
    if (lane == 0) R[i + (int64_t)(j + 1) * ldr] = r;
  }
}

template <int V, int kPanel>
__device__ int cgs_body(const SweepArgs& a, const int G, const int b, double* smem, uint64_t* s_full,
                        uint64_t* s_empty, int* s_flags) {
  const int n = a.n;
  const int chunk = a.chunk;
  double* s_piece = smem;                          // kWarps x kPieceCols warp partials
  double* s_dacc = s_piece + kWarps * kPieceCols;  // CTA partials of the next column (staged mode)
  double* s_rcol = s_dacc + n;                     // r_{i,j}, i < j, of the current column
  double* s_rnext = s_rcol + n;                    // r_{i,j+1} being assembled
  double* s_buf = s_rnext + n;                     // kThreads + 1 reduction scratch
  double* s_scal = s_buf + kThreads + 1;           // r_jj, 1/r_jj, status
  double* s_xtmp = s_scal + 8;                     // chunk rows (long-row MVs, resident mode)
  // a.stages pivot buffers of 2 * chunk doubles, 128-byte aligned (bulk
  // copies need 16): the offset is rounded up to 16 doubles.
  double* s_ring = smem + ((s_xtmp + chunk - smem + 15) & ~(int64_t)15);

  const int tid = threadIdx.x;
  const int64_t m = a.m;
  const int64_t rpc = a.rpc;
  const int64_t k0 = (int64_t)b * rpc;
  const int64_t k1 = (k0 + rpc < m) ? k0 + rpc : m;
  const int crows_all = (int)(k1 - k0);
  const bool resident = rpc <= chunk;
  const bool warp_rows = a.mv_warp != 0;
  const int32_t* __restrict__ rowptr = a.rowptr;
  const int32_t* __restrict__ colidx = a.col;
  const double* __restrict__ val = a.val;
  const double* __restrict__ Z = a.Z;
  double* __restrict__ Q = a.Q;
  double* __restrict__ X = a.X;
  double* __restrict__ R = a.R;
  const int64_t ldz = a.ldz, ldq = a.ldq, ldx = a.ldx;
  const int ldr = a.ldr;
  double* W = X;         // HA / naive: the gathered copy of z_j
  double* XS = X + ldx;  // HA / naive, staged: x_j
  // Block (j, b) of qp: q_j then p_j on this CTA's rows, rpc doubles each.
  double* qp_cta = a.qp + (int64_t)b * 2 * rpc;
  const int64_t cta_stride = (int64_t)G * 2 * rpc;  // from pivot j to j+1
  double* part_norm = a.part + 2 * (int64_t)n * G;
  unsigned int gen = 0;

  PivotRing ring;
  ring.full = s_full;
  ring.empty = s_empty;
  ring.buf = s_ring;
  ring.S = a.stages;
  ring.chunk = chunk;
  ring.next = 0;
  ring.issued = 0;
  ring.abort = s_flags + 2;
  if (tid == 0) {
    s_flags[2] = 0;
    for (int s = 0; s < ring.S; ++s) {
      mbar_init(&s_full[s], 1);
      mbar_init(&s_empty[s], kWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }

  // Phase 0: R = 0; HP: X = A Z on own rows (one block product).
  if (b == 0) {
    for (int64_t t = tid; t < (int64_t)n * n; t += kThreads) R[(t % n) + (t / n) * ldr] = 0.0;
  }
  if (V == kHP) (void)spmm_slab_panel<kPanel>(rowptr, colidx, val, Z, ldz, X, ldx, nullptr, 0, k0, k1, n, warp_rows);
  __syncthreads();

  // Resident slots: z_j, x_j of the current column and z_{j+1}^{(0)}.
  double zr[kResRows], xr[kResRows], z1r[kResRows];
  if (resident) load_slots(Z, k0, crows_all, zr);

  for (int j = 0; j < n; ++j) {
    const int cur = j & 1;
    double* part_cur = a.part + (int64_t)cur * n * G;  // CTA partials of column j+1's coefficients
    const bool has_next = j + 1 < n;
    const double* z1col = has_next ? Z + (int64_t)(j + 1) * ldz : nullptr;

    // ---------------- U: z_j (HP: x_j) and the next column's dots ----------------
    CGS_TRACE(j, 0);
    double sl = 0.0;
    if (resident) {
      if (V == kHP) load_slots(X + (int64_t)j * ldx, k0, crows_all, xr);
      load_slots(z1col, k0, crows_all, z1r);
      if (!update_pass<V>(j, crows_all, qp_cta, cta_stride, rpc, 0, s_rcol, ring, zr, xr, z1r,
                          has_next ? part_cur + (int64_t)b * n : nullptr, false, s_piece)) {
        if (tid == 0) set_status(a.ctl, kDevTimeout, -1);
        return body_result(kDevTimeout, 0);
      }
#pragma unroll
      for (int t = 0; t < kResRows; ++t) {
        const int rr = tid + t * kThreads;
        if (rr < crows_all) {
          if (V == kHP) sl = fma(zr[t], xr[t], sl);
          else W[k0 + rr] = zr[t];
        }
      }
    } else {
      for (int64_t c0 = k0; c0 < k1; c0 += chunk) {
        const int crows = (int)((k1 - c0) < chunk ? (k1 - c0) : chunk);
        load_slots(Z + (int64_t)j * ldz, c0, crows, zr);
        if (V == kHP) load_slots(X + (int64_t)j * ldx, c0, crows, xr);
        load_slots(z1col, c0, crows, z1r);
        if (!update_pass<V>(j, crows, qp_cta, cta_stride, rpc, c0 - k0, s_rcol, ring, zr, xr, z1r,
                            has_next ? s_dacc : nullptr, c0 > k0, s_piece)) {
          if (tid == 0) set_status(a.ctl, kDevTimeout, -1);
          return body_result(kDevTimeout, 0);
        }
        double* zdst = (V == kHP) ? Q + (int64_t)j * ldq : W;
#pragma unroll
        for (int t = 0; t < kResRows; ++t) {
          const int rr = tid + t * kThreads;
          if (rr < crows) {
            zdst[c0 + rr] = zr[t];
            if (V == kHP) {
              X[c0 + rr + (int64_t)j * ldx] = xr[t];
              sl = fma(zr[t], xr[t], sl);
            }
          }
        }
      }
      if (has_next)
        for (int i = tid; i < j; i += kThreads) part_cur[(int64_t)b * n + i] = s_dacc[i];
    }

    // ---------------- MV (HA, naive) and the diagonal ----------------
    CGS_TRACE(j, 1);
    if (V == kHP) {
      sl = block_sum(sl, s_buf);
      if (tid == 0) part_norm[b] = sl;
      if (!sync_all<false>(a.ctl, gen, (unsigned)G, s_flags)) return body_result(kDevTimeout, 0);
    } else {
      if (!sync_all<false>(a.ctl, gen, (unsigned)G, s_flags)) return body_result(kDevTimeout, 0);  // z_j complete in W
      CGS_TRACE(j, 2);
      sl = mv_rows(rowptr, colidx, val, W, 1.0, false, k0, k1, resident, warp_rows, xr, zr, XS, s_xtmp, true);
      sl = block_sum(sl, s_buf);
      if (tid == 0) part_norm[b] = sl;
      CGS_TRACE(j, 3);
      sync_arrive<false>(a.ctl, gen, s_flags);
      // r_{i,j+1}, i < j: their partials were stored before the previous wait.
      if (has_next && j > 0) sum_assigned(part_cur, G, n, j, R, ldr, b);
      if (!sync_wait<false>(a.ctl, gen, (unsigned)G, s_flags)) return body_result(kDevTimeout, 0);
    }
    CGS_TRACE(j, 4);
    // HP: r_{i,j+1}, i < j (partials stored before the norm wait), while warp 0
    // forms r_jj.
    if (V == kHP && has_next && j > 0) sum_assigned(part_cur, G, n, j, R, ldr, b);
    diagonal(part_norm, G, s_scal);
    CGS_TRACE(j, 5);
    if (s_scal[2] != 0.0) return body_result((int)s_scal[2], j + 1);  // the same verdict in every CTA
    const double inv = s_scal[1];
    if (b == 0 && tid == 0) R[j + (int64_t)j * ldr] = s_scal[0];

    // ---------------- MV2 (naive) and F ----------------
    double dj = 0.0;
    double* qj = Q + (int64_t)j * ldq;
    double* qpq = qp_cta + (int64_t)j * cta_stride;  // this CTA's block of pivot j
    double* qpp = qpq + rpc;
    if (resident) {
      // naive: p_j = A q_j with q_j = z_j / r_jj gathered on the fly (into xr)
      if (V == kNaive)
        (void)mv_rows(rowptr, colidx, val, W, inv, true, k0, k1, true, warp_rows, xr, zr, nullptr, s_xtmp, false);
#pragma unroll
      for (int t = 0; t < kResRows; ++t) {
        const int rr = tid + t * kThreads;
        if (rr < crows_all) {
          const double qv = zr[t] * inv;
          const double pv = (V == kNaive) ? xr[t] : xr[t] * inv;
          qj[k0 + rr] = qv;
          qpq[rr] = qv;
          qpp[rr] = pv;
          dj = fma(pv, z1r[t], dj);
        }
      }
    } else {
      double* pbuf = (V == kHP) ? X + (int64_t)j * ldx : XS;  // x_j of the staged pass
      if (V == kNaive) {
        (void)mv_rows(rowptr, colidx, val, W, inv, true, k0, k1, false, warp_rows, xr, zr, pbuf, s_xtmp, false);
        __syncthreads();  // p_j rows are read below by other threads than wrote them
      }
      const double* zsrc = (V == kHP) ? qj : W;
      for (int64_t k = k0 + tid; k < k1; k += kThreads) {
        const double qv = zsrc[k] * inv;
        const double pv = (V == kNaive) ? pbuf[k] : pbuf[k] * inv;
        qj[k] = qv;
        qpq[k - k0] = qv;
        qpp[k - k0] = pv;
        if (has_next) dj = fma(pv, z1col[k], dj);
      }
    }
    fence_proxy_async_global();  // the block of pivot j is read by bulk copies from the next column on
    CGS_TRACE(j, 6);
    if (!has_next) break;
    dj = block_sum(dj, s_buf);
    if (tid == 0) part_cur[(int64_t)b * n + j] = dj;
    CGS_TRACE(j, 7);

    // ---------------- r_{:,j+1} ----------------
    if (!sync_all<false>(a.ctl, gen, (unsigned)G, s_flags)) return body_result(kDevTimeout, 0);
    CGS_TRACE(j, 8);
    if (tid < 32) {
      const double r = warp0_sum_ctas(part_cur + j, n, G);
      if (tid == 0) {
        s_rnext[j] = r;
        if (b == 0) R[j + (int64_t)(j + 1) * ldr] = r;
      }
    } else {
      // r_{i,j+1}, i < j, summed by their CTAs into R before this wait
      for (int i = tid - 32; i < j; i += kThreads - 32) s_rnext[i] = ld_cg(R + i + (int64_t)(j + 1) * ldr);
    }
    __syncthreads();
    CGS_TRACE(j, 9);
    double* t = s_rcol;
    s_rcol = s_rnext;
    s_rnext = t;
    if (resident) {
#pragma unroll
      for (int s = 0; s < kResRows; ++s) zr[s] = z1r[s];  // z_{j+1}^{(0)}
    }
  }
  return 0;
}

template <int V, int kPanel>
__global__ void __launch_bounds__(kThreads, 1) cgs_sweep_kernel(const SweepArgs a) {
  extern __shared__ __align__(16) double smem[];
  __shared__ __align__(8) uint64_t s_full[kCgsMaxStages];
  __shared__ __align__(8) uint64_t s_empty[kCgsMaxStages];
  __shared__ int s_flags[3];  // barrier scratch (2), ring abort flag
  const int r = cgs_body<V, kPanel>(a, gridDim.x, blockIdx.x, smem, s_full, s_empty, s_flags);
  if (r != 0 && (r >> 24) != kDevTimeout && blockIdx.x == 0 && threadIdx.x == 0) set_status(a.ctl, r >> 24, r & 0xFFFFFF);
}

}  // namespace

// naive and HA have no block product; HP has one kernel per panel width.
static const void* cgs_fn(int variant, int panel = 8) {
  switch (variant) {
    case kNaive: return reinterpret_cast<const void*>(cgs_sweep_kernel<kNaive, 8>);
    case kHA: return reinterpret_cast<const void*>(cgs_sweep_kernel<kHA, 8>);
    default:
      return panel == 4 ? reinterpret_cast<const void*>(cgs_sweep_kernel<kHP, 4>)
                        : reinterpret_cast<const void*>(cgs_sweep_kernel<kHP, 8>);
  }
}

// Everything but the pivot buffers, in doubles, with the padding that
// aligns the first buffer to 16 doubles.
static size_t cgs_fixed_doubles(int n, int chunk) {
  const size_t used = (size_t)kWarps * kPieceCols + 3 * (size_t)n + kThreads + 1 + 8 + (size_t)chunk;
  return (used + 15) & ~(size_t)15;
}

cudaError_t cgs_smem_plan(int variant, int n, int chunk, int* stages, size_t* smem) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
  cudaFuncAttributes fa;
  if ((e = cudaFuncGetAttributes(&fa, cgs_fn(variant))) != cudaSuccess) return e;
  const size_t avail = (size_t)optin - fa.sharedSizeBytes;
  const size_t fixed = sizeof(double) * cgs_fixed_doubles(n, chunk);
  const size_t per = sizeof(double) * 2 * (size_t)chunk;
  int s = avail > fixed ? (int)((avail - fixed) / per) : 0;
  if (s > kCgsMaxStages) s = kCgsMaxStages;
  if (s < 2) return cudaErrorInvalidValue;
  *stages = s;
  *smem = fixed + per * (size_t)s;
  return cudaSuccess;
}

cudaError_t cgs_prepare(int device) {
  int optin = 0;
  cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  if (e != cudaSuccess) return e;
  const int instances[4][2] = {{kNaive, 8}, {kHA, 8}, {kHP, 8}, {kHP, 4}};
  for (const auto& k : instances) {
    const void* fn = cgs_fn(k[0], k[1]);
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, fn)) != cudaSuccess) return e;
    const int dyn = optin - (int)fa.sharedSizeBytes;
    if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t cgs_max_ctas(int variant, size_t smem, int* max_ctas) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cgs_fn(variant), kThreads, smem)) != cudaSuccess)
    return e;
  *max_ctas = sms * per_sm;
  return cudaSuccess;
}

cudaError_t cgs_launch(int variant, const SweepArgs& a, int grid, size_t smem, cudaStream_t s) {
  SweepArgs copy = a;
  void* args[] = {&copy};
  return cudaLaunchCooperativeKernel(cgs_fn(variant, a.spmm_panel), dim3(grid), dim3(kThreads), args, smem, s);
}

}  // namespace mgsa
