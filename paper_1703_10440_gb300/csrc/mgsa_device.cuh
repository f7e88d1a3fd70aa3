// Device helpers shared by the MGS and CGS kernels of libmgsa: mbarrier and
// bulk-copy primitives, device-wide split barrier with bounded waits,
// deterministic block and grid reductions,
// the diagonal r_jj = sqrt(z_j^T x_j) with its breakdown verdict, CSR row
// products and the block product X = A Z.  Each including translation unit
// gets its own copy (anonymous namespace).
#pragma once
#include "mgsa_internal.cuh"

namespace mgsa {

namespace {


__device__ __forceinline__ unsigned long long global_timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_relaxed_i32(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// ---- mbarrier and bulk-copy primitives (PTX ISA: mbarrier, cp.async.bulk) ----

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// Waits for the completion of the phase of `bar` with parity `parity`.
// False once kSpinLimitNs have passed (then *abort is raised for the whole
// CTA) or as soon as another thread of the CTA has raised *abort.
__device__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_timer_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort) return false;
    if (global_timer_ns() - t0 > kSpinLimitNs) {
      *abort = 1;
      return false;
    }
  }
}

// bytes (a multiple of 16, both addresses 16-byte aligned) from global to
// this CTA's shared memory; completion is counted on `bar`.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

// Makes this thread's earlier generic-proxy global stores visible to later
// bulk copies (async proxy) that read them.
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// Plain loads that bypass L1: data written by other CTAs during this kernel.
__device__ __forceinline__ double ld_cg(const double* p) { return __ldcg(p); }

__device__ __forceinline__ double warp_sum(double v) {
  // Butterfly: every lane ends with the same value (each pairwise sum is the
  // same two operands in every lane, and + is commutative).
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic CTA-wide sum returned to every thread: the 512 values go to
// shared memory, lane l of warp 0 adds values l, l+32, ... in order, then a
// butterfly.  (21 warp-wide FP64 instructions instead of 85 for 16 butterflies.)
__device__ double block_sum(double v, double* s_buf) {
  s_buf[threadIdx.x] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = s_buf[threadIdx.x];
#pragma unroll
    for (int w = 1; w < kWarps; ++w) t += s_buf[threadIdx.x + 32 * w];
    t = warp_sum(t);
    if (threadIdx.x == 0) s_buf[kThreads] = t;
  }
  __syncthreads();
  const double r = s_buf[kThreads];
  __syncthreads();
  return r;
}

__device__ void set_status(int* ctl, int code, int column) {
  if (atomicCAS(&ctl[kCtlStatus], 0, code) == 0) atomicExch(&ctl[kCtlColumn], column);
}

// Device-wide barrier for a cooperative launch, in two halves so that a CTA
// can do independent work between arriving and waiting.  The counter only
// grows during a launch (it is zeroed before each launch): barrier number k
// (k = 1, 2, ...) is passed once it reaches k times the number of CTAs that
// take part (the grid, or one gang of CTAs of a grouped launch).  Arrival is a
// fire-and-forget release reduction; every CTA then polls the counter with
// acquire loads.  Only thread 0 of a CTA touches it; `gen` (the number of
// barriers passed) is meaningful in thread 0 only.
__device__ __forceinline__ void grid_arrive(int* ctl, unsigned int gen, int* s_unused) {
  (void)gen;
  (void)s_unused;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int* count = reinterpret_cast<unsigned int*>(&ctl[kCtlBarCount]);
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(count) : "memory");
  }
}

// Returns false if the wait ran past kSpinLimitNs or another CTA already
// recorded a failure (then every CTA leaves the kernel).  `nctas`: the CTAs
// that arrive at this barrier (the whole grid, or one gang of a grouped launch).
__device__ bool grid_wait(int* ctl, unsigned int& gen, unsigned int nctas, int* s_ok) {
  if (threadIdx.x == 0) {
    const unsigned int* count = reinterpret_cast<const unsigned int*>(&ctl[kCtlBarCount]);
    const unsigned int target = (gen + 1u) * nctas;
    int ok = 1;
    if (ld_acquire_u32(count) < target) {
      const unsigned long long t0 = global_timer_ns();
      unsigned int polls = 0;
      while (ld_acquire_u32(count) < target) {
        if ((++polls & 255u) == 0u) {
          if (ld_relaxed_i32(&ctl[kCtlStatus]) != 0) { ok = 0; break; }
          if (global_timer_ns() - t0 > kSpinLimitNs) {
            set_status(ctl, kDevTimeout, -1);
            ok = 0;
            break;
          }
        }
      }
    }
    gen += 1u;
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

__device__ __forceinline__ bool grid_sync(int* ctl, unsigned int& gen, unsigned int nctas, int* s_flags) {
  grid_arrive(ctl, gen, s_flags);
  return grid_wait(ctl, gen, nctas, s_flags + 1);
}

// Hardware barrier of a thread-block cluster: every thread of every CTA of
// the cluster arrives (release) and waits (acquire), so the memory writes
// before it are visible to the whole cluster after it.  No spinning: the
// hardware holds the warps.
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

// Synchronisation of the step body: device-wide for the single-instance
// kernel, CTA-wide when one CTA owns a whole instance (batched kernel),
// cluster-wide when one thread-block cluster owns it (kCluster).
// The cluster form keeps the CTA barrier in front of the arrive, as
// grid_arrive does: the work between arrive and wait may reuse shared buffers
// that other threads of the CTA read just before.
template <bool kBatch, bool kCluster = false>
__device__ __forceinline__ void sync_arrive(int* ctl, unsigned int gen, int* s_flags) {
  if (kCluster) {
    __syncthreads();
    cluster_arrive();
  } else if (kBatch) __syncthreads();
  else grid_arrive(ctl, gen, s_flags);
}

// `nctas`: CTAs taking part in a device-wide barrier (unused for the CTA and
// cluster forms).
template <bool kBatch, bool kCluster = false>
__device__ __forceinline__ bool sync_wait(int* ctl, unsigned int& gen, unsigned int nctas, int* s_flags) {
  if (kCluster) {
    cluster_wait();
    return true;
  }
  if (kBatch) {
    __syncthreads();
    return true;
  }
  return grid_wait(ctl, gen, nctas, s_flags + 1);
}

template <bool kBatch, bool kCluster = false>
__device__ __forceinline__ bool sync_all(int* ctl, unsigned int& gen, unsigned int nctas, int* s_flags) {
  sync_arrive<kBatch, kCluster>(ctl, gen, s_flags);
  return sync_wait<kBatch, kCluster>(ctl, gen, nctas, s_flags);
}

// Result of the step body: 0, or (device status << 24) | 1-based column.
__device__ __forceinline__ int body_result(int status, int column) { return (status << 24) | (column & 0xFFFFFF); }

// Sum over CTAs b (fixed tree) of part[b * stride], by one warp: lane l adds
// the CTAs l, l + 32, ..., l + 128 of each group of 160 in that order, then a
// butterfly.  Every lane returns the sum.
__device__ __forceinline__ double warp_sum_ctas(const double* part, int64_t stride, int G, int lane) {
  double t = 0.0;
  for (int b0 = 0; b0 < G; b0 += 160) {
    double v[5];
#pragma unroll
    for (int s = 0; s < 5; ++s) {
      const int bb = b0 + lane + 32 * s;
      v[s] = bb < G ? ld_cg(part + bb * stride) : 0.0;
    }
    t += (((v[0] + v[1]) + v[2]) + v[3]) + v[4];
  }
  return warp_sum(t);
}

// The same sum by warp 0 (lane = threadIdx.x).
__device__ __forceinline__ double warp0_sum_ctas(const double* part, int64_t stride, int G) {
  return warp_sum_ctas(part, stride, G, (int)threadIdx.x);
}

// r_ii from the norm partials: one thread forms the sum's square root, its
// reciprocal and the breakdown verdict and broadcasts them.
// s_scal[0] = r_ii, s_scal[1] = 1/r_ii, s_scal[2] = status (0 ok).
__device__ void diagonal(const double* part_norm, int G, double* s_scal) {
  if (threadIdx.x < 32) {
    const double stot = warp0_sum_ctas(part_norm, 1, G);
    if (threadIdx.x == 0) {
      int st = kDevOk;
      double r = 0.0, inv = 0.0;
      if (isnan(stot) || isinf(stot)) st = kDevNonfinite;
      else if (!(stot > 0.0)) st = kDevBreakdown;
      else {
        r = sqrt(stot);
        inv = 1.0 / r;
      }
      s_scal[0] = r;
      s_scal[1] = inv;
      s_scal[2] = (double)st;
    }
  }
  __syncthreads();
}

// The same verdict from a sum every thread already holds (one CTA per instance).
__device__ void diagonal_of(double stot, double* s_scal) {
  if (threadIdx.x == 0) {
    int st = kDevOk;
    double r = 0.0, inv = 0.0;
    if (isnan(stot) || isinf(stot)) st = kDevNonfinite;
    else if (!(stot > 0.0)) st = kDevBreakdown;
    else {
      r = sqrt(stot);
      inv = 1.0 / r;
    }
    s_scal[0] = r;
    s_scal[1] = inv;
    s_scal[2] = (double)st;
  }
  __syncthreads();
}

// out[j] = the sum over CTAs b (in the order of b) of part[b * stride + j] for
// j in [jbeg, jend), lane per j: warp w adds the partials of the CTAs in
// [w*G/16, (w+1)*G/16) in order, then warp 0 adds the 16 warp sums in order.
// Loads are coalesced because part is laid out [CTA][slot].  When rdst is set,
// the sum for j is also stored at rdst[(j - roff) * rstride] (a row or a
// column of R).
__device__ void reduce_range(const double* part, int G, int stride, int jbeg, int jend, double* out, double* s_buf,
                             double* rdst, int64_t rstride, int roff) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int bb0 = (int)((int64_t)G * warp / kWarps), bb1 = (int)((int64_t)G * (warp + 1) / kWarps);
  for (int j0 = jbeg; j0 < jend; j0 += 32) {
    const int j = j0 + lane;
    double t0 = 0.0, t1 = 0.0;
    int bb = bb0;
    for (; bb + 1 < bb1; bb += 2) {
      const double v0 = j < jend ? ld_cg(part + (int64_t)bb * stride + j) : 0.0;
      const double v1 = j < jend ? ld_cg(part + (int64_t)(bb + 1) * stride + j) : 0.0;
      t0 += v0;
      t1 += v1;
    }
    if (bb < bb1) t0 += j < jend ? ld_cg(part + (int64_t)bb * stride + j) : 0.0;
    s_buf[threadIdx.x] = t0 + t1;
    __syncthreads();
    if (warp == 0 && j < jend) {
      double t = s_buf[lane];
#pragma unroll
      for (int w = 1; w < kWarps; ++w) t += s_buf[lane + 32 * w];
      out[j] = t;
      if (rdst) rdst[(int64_t)(j - roff) * rstride] = t;
    }
    __syncthreads();
  }
}

constexpr int kResRows = kMaxChunk / kThreads;  // rows per thread when a CTA's slab is one chunk

// out[q] = sum_e val[e] * (scale_src ? src[col[e]] * scale : src[col[e]]) for
// the rows k + q*kThreads (q < kRows) below k1, each summed in stored order.
// The kRows rows advance in lockstep so that their gathers are in flight
// together (each entry is two dependent loads: the column index, then the
// gathered value; loading the next entry's index ahead, as the block product
// does, measured slower here: 3D naive 81.4 -> 85.3 ms).  kL1: gather through L1 (only for a source vector this SM
// has not read earlier in the launch at the gathered addresses), else from L2.
template <int kRows, bool kL1 = false>
__device__ __forceinline__ void csr_rows(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                                         const double* __restrict__ val, const double* src, double scale,
                                         bool scale_src, int64_t k, int64_t k1, double out[kRows]) {
  int e[kRows], e1[kRows];
#pragma unroll
  for (int q = 0; q < kRows; ++q) {
    const int64_t kk = k + q * kThreads;
    e[q] = kk < k1 ? __ldg(rowptr + kk) : 0;
    e1[q] = kk < k1 ? __ldg(rowptr + kk + 1) : 0;
    out[q] = 0.0;
  }
  for (;;) {
    bool any = false;
#pragma unroll
    for (int q = 0; q < kRows; ++q) any |= e[q] < e1[q];
    if (!any) break;
#pragma unroll
    for (int q = 0; q < kRows; ++q) {
      if (e[q] < e1[q]) {
        const double* g = src + __ldg(colidx + e[q]);
        const double zv = kL1 ? __ldca(g) : ld_cg(g);
        out[q] = fma(__ldg(val + e[q]), scale_src ? zv * scale : zv, out[q]);
        ++e[q];
      }
    }
  }
}

// The same sums with each row's entries taken kE at a time: the kE column
// indices and values of a row first, then their kE gathers, then the FMAs in
// stored order (the same order as csr_rows, so the same bits).  More loads in
// flight per row, more registers.
template <int kRows, int kE, bool kL1 = false>
__device__ __forceinline__ void csr_rows_e(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                                           const double* __restrict__ val, const double* src, double scale,
                                           bool scale_src, int64_t k, int64_t k1, double out[kRows]) {
  int e[kRows], e1[kRows];
#pragma unroll
  for (int q = 0; q < kRows; ++q) {
    const int64_t kk = k + q * kThreads;
    e[q] = kk < k1 ? __ldg(rowptr + kk) : 0;
    e1[q] = kk < k1 ? __ldg(rowptr + kk + 1) : 0;
    out[q] = 0.0;
  }
  for (;;) {
    bool any = false;
#pragma unroll
    for (int q = 0; q < kRows; ++q) any |= e[q] < e1[q];
    if (!any) break;
    int c[kRows][kE];
    double v[kRows][kE], g[kRows][kE];
#pragma unroll
    for (int q = 0; q < kRows; ++q)
#pragma unroll
      for (int t = 0; t < kE; ++t) {
        const bool ok = e[q] + t < e1[q];
        c[q][t] = ok ? __ldg(colidx + e[q] + t) : 0;
        v[q][t] = ok ? __ldg(val + e[q] + t) : 0.0;
      }
#pragma unroll
    for (int q = 0; q < kRows; ++q)
#pragma unroll
      for (int t = 0; t < kE; ++t) {
        const double* a = src + c[q][t];
        g[q][t] = e[q] + t < e1[q] ? (kL1 ? __ldca(a) : ld_cg(a)) : 0.0;
      }
#pragma unroll
    for (int q = 0; q < kRows; ++q) {
#pragma unroll
      for (int t = 0; t < kE; ++t)
        if (e[q] + t < e1[q]) out[q] = fma(v[q][t], scale_src ? g[q][t] * scale : g[q][t], out[q]);
      e[q] += kE;
    }
  }
}

// csr_rows with the source vector in this CTA's shared memory, indexed by
// the column itself: for a CTA that owns every row of its instance (the
// batched kernel), so that each entry costs one dependent global load (its
// column index) instead of two.  Same operations in the same order as
// csr_rows, so the same bits.
template <int kRows>
__device__ __forceinline__ void csr_rows_sh(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                                            const double* __restrict__ val, const double* s_src, int64_t k, int64_t k1,
                                            double out[kRows]) {
  int e[kRows], e1[kRows];
#pragma unroll
  for (int q = 0; q < kRows; ++q) {
    const int64_t kk = k + q * kThreads;
    e[q] = kk < k1 ? __ldg(rowptr + kk) : 0;
    e1[q] = kk < k1 ? __ldg(rowptr + kk + 1) : 0;
    out[q] = 0.0;
  }
  for (;;) {
    bool any = false;
#pragma unroll
    for (int q = 0; q < kRows; ++q) any |= e[q] < e1[q];
    if (!any) break;
#pragma unroll
    for (int q = 0; q < kRows; ++q) {
      if (e[q] < e1[q]) {
        out[q] = fma(__ldg(val + e[q]), s_src[__ldg(colidx + e[q])], out[q]);
        ++e[q];
      }
    }
  }
}

__device__ __forceinline__ void csr_rows4(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                                          const double* __restrict__ val, const double* src, double scale,
                                          bool scale_src, int64_t k, int64_t k1, double out[4]) {
  csr_rows<4>(rowptr, colidx, val, src, scale, scale_src, k, k1, out);
}

// Long rows: one warp per row.  Lane l takes the entries e0 + l, e0 + l + 32,
// ... (coalesced column and value loads), two accumulators, then a butterfly;
// every lane returns the row's sum (a fixed tree, so deterministic).  kL1 as
// for csr_rows.
template <bool kL1 = false>
__device__ __forceinline__ double csr_row_warp(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                                               const double* __restrict__ val, const double* src, double scale,
                                               bool scale_src, int64_t k) {
  const int lane = threadIdx.x & 31;
  const int e0 = __ldg(rowptr + k), e1 = __ldg(rowptr + k + 1);
  double acc0 = 0.0, acc1 = 0.0;
  int e = e0 + lane;
  for (; e + 32 < e1; e += 64) {
    const double* a0 = src + __ldg(colidx + e);
    const double* a1 = src + __ldg(colidx + e + 32);
    const double g0 = kL1 ? __ldca(a0) : ld_cg(a0);
    const double g1 = kL1 ? __ldca(a1) : ld_cg(a1);
    acc0 = fma(__ldg(val + e), scale_src ? g0 * scale : g0, acc0);
    acc1 = fma(__ldg(val + e + 32), scale_src ? g1 * scale : g1, acc1);
  }
  if (e < e1) {
    const double* a0 = src + __ldg(colidx + e);
    const double g0 = kL1 ? __ldca(a0) : ld_cg(a0);
    acc0 = fma(__ldg(val + e), scale_src ? g0 * scale : g0, acc0);
  }
  return warp_sum(acc0 + acc1);
}

// The thread-per-row part of spmm_slab_panel: kSR rows per thread in
// lockstep, each row summed in stored order (so the sums do not depend on
// kSR).  Returns this thread's share of z_0^T x_0, its rows in ascending order.
template <int kPanel, int kSR>
__device__ double spmm_rows(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                            const double* __restrict__ val, const double* __restrict__ Z, int64_t ldz,
                            double* __restrict__ X, int64_t ldx, double* __restrict__ Q, int64_t ldq, int64_t k0,
                            int64_t k1, int n) {
  const int tid = threadIdx.x;
  double s0 = 0.0;
  for (int64_t kb = k0 + tid; kb < k1; kb += kSR * kThreads) {
    int eb[kSR], ee[kSR];
#pragma unroll
    for (int q = 0; q < kSR; ++q) {
      const int64_t kk = kb + q * kThreads;
      eb[q] = kk < k1 ? __ldg(rowptr + kk) : 0;
      ee[q] = kk < k1 ? __ldg(rowptr + kk + 1) : 0;
    }
    for (int j0 = 0; j0 < n; j0 += kPanel) {
      const int w = (n - j0) < kPanel ? (n - j0) : kPanel;
      double acc[kSR][kPanel];
      int e[kSR];
      // Column index and value of each row's next entry, loaded one entry
      // ahead so that an entry's gathers wait for one load, not two.
      int cn[kSR];
      double vn[kSR];
#pragma unroll
      for (int q = 0; q < kSR; ++q) {
        e[q] = eb[q];
        cn[q] = e[q] < ee[q] ? __ldg(colidx + e[q]) : 0;
        vn[q] = e[q] < ee[q] ? __ldg(val + e[q]) : 0.0;
#pragma unroll
        for (int jj = 0; jj < kPanel; ++jj) acc[q][jj] = 0.0;
      }
      for (;;) {
        bool any = false;
#pragma unroll
        for (int q = 0; q < kSR; ++q) any |= e[q] < ee[q];
        if (!any) break;
#pragma unroll
        for (int q = 0; q < kSR; ++q) {
          if (e[q] < ee[q]) {
            const double v = vn[q];
            const double* zc = Z + cn[q] + (int64_t)j0 * ldz;
            if (e[q] + 1 < ee[q]) {
              cn[q] = __ldg(colidx + e[q] + 1);
              vn[q] = __ldg(val + e[q] + 1);
            }
#pragma unroll
            for (int jj = 0; jj < kPanel; ++jj)
              if (jj < w) acc[q][jj] = fma(v, __ldg(zc + jj * ldz), acc[q][jj]);
            ++e[q];
          }
        }
      }
#pragma unroll
      for (int q = 0; q < kSR; ++q) {
        const int64_t kk = kb + q * kThreads;
        if (kk < k1) {
#pragma unroll
          for (int jj = 0; jj < kPanel; ++jj) {
            if (jj < w) {
              const double zk = __ldg(Z + kk + (int64_t)(j0 + jj) * ldz);
              X[kk + (int64_t)(j0 + jj) * ldx] = acc[q][jj];
              if (Q) Q[kk + (int64_t)(j0 + jj) * ldq] = zk;
              if (j0 + jj == 0) s0 = fma(zk, acc[q][0], s0);
            }
          }
        }
      }
    }
  }
  return s0;
}

// X = A Z on the rows [k0, k1) for the n columns of Z (the block product of
// Algorithms 6 and 8), kPanel columns at a time so that one pass over a row's
// entries serves kPanel columns.  Long rows (warp_rows): one warp per row,
// lanes split the row's entries, one butterfly per column.  Otherwise two or
// four rows per thread in lockstep (spmm_rows), each row summed in stored
// order.  When Q is set, Q = Z on the same rows.  Returns this thread's share
// of z_0^T x_0.  Every column's sums are the same for any panel width.
template <int kPanel>
__device__ double spmm_slab_panel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                                  const double* __restrict__ val, const double* __restrict__ Z, int64_t ldz,
                                  double* __restrict__ X, int64_t ldx, double* __restrict__ Q, int64_t ldq,
                                  int64_t k0, int64_t k1, int n, bool warp_rows) {
  const int tid = threadIdx.x;
  double s0 = 0.0;
  if (warp_rows) {
    const int lane = tid & 31, warp = tid >> 5;
    for (int64_t k = k0 + warp; k < k1; k += kWarps) {
      const int e0 = __ldg(rowptr + k), e1 = __ldg(rowptr + k + 1);
      for (int j0 = 0; j0 < n; j0 += kPanel) {
        const int w = (n - j0) < kPanel ? (n - j0) : kPanel;
        double acc[kPanel];
#pragma unroll
        for (int jj = 0; jj < kPanel; ++jj) acc[jj] = 0.0;
        for (int e = e0 + lane; e < e1; e += 32) {
          const double v = __ldg(val + e);
          const double* zc = Z + __ldg(colidx + e) + (int64_t)j0 * ldz;
#pragma unroll
          for (int jj = 0; jj < kPanel; ++jj)
            if (jj < w) acc[jj] = fma(v, __ldg(zc + jj * ldz), acc[jj]);
        }
#pragma unroll
        for (int jj = 0; jj < kPanel; ++jj) {
          if (jj < w) {
            const double x = warp_sum(acc[jj]);
            if (lane == jj) {
              const double zk = __ldg(Z + k + (int64_t)(j0 + jj) * ldz);
              X[k + (int64_t)(j0 + jj) * ldx] = x;
              if (Q) Q[k + (int64_t)(j0 + jj) * ldq] = zk;
              if (j0 + jj == 0) s0 = fma(zk, x, s0);
            }
          }
        }
      }
    }
    return s0;
  }
  // Two rows per thread per round on slabs of more than 4 x kThreads rows
  // (fewer live registers, more loads in flight: 3D 128^3 HP 98.89 -> 98.22
  // ms), four on smaller ones (a 1728-row slab would leave the second of two
  // rounds part idle: Poisson 512^2 HP 3.814 -> 3.825 ms with two).
  if (k1 - k0 > 4 * kThreads) return spmm_rows<kPanel, 2>(rowptr, colidx, val, Z, ldz, X, ldx, Q, ldq, k0, k1, n);
  return spmm_rows<kPanel, 4>(rowptr, colidx, val, Z, ldz, X, ldx, Q, ldq, k0, k1, n);
}

}  // namespace

}  // namespace mgsa
