// Single-instance A-inner-product MGS: one persistent cooperative kernel runs
// the whole right-looking loop (Algorithms 4, 7, 8 of Imakura & Yamamoto,
// arXiv 1703.10440) over row slabs owned by the CTAs.
//
// Every CTA owns rows [b*rpc, min(m, (b+1)*rpc)) of Z/Q and X for the whole
// kernel.  Step i of the loop is:
//
//   L  (i > 0)  update column i with step i-1:  z_i -= r_{i-1,i} q_{i-1}
//               (HP also x_i -= r_{i-1,i} p_{i-1}); HP accumulates z_i^T x_i.
//   MV  (HA, naive) x_i = A z_i  (eq. in Algorithms 4/7), accumulating z_i^T x_i.
//   D   r_ii = sqrt(sum of partials)  (breakdown / non-finite check).
//   MV2 (naive) p_i = A q_i  with q_i = z_i / r_ii gathered on the fly.
//   B   q_i = z_i / r_ii (stored), p_i = x_i / r_ii (eq. (tec1)); for every
//       j > i: apply step i-1's rank-1 updates z_j -= r_{i-1,j} q_{i-1}
//       (HP: x_j -= r_{i-1,j} p_{i-1}, eq. (tec2) one term at a time) and
//       accumulate r_ij = p_i^T z_j^{(i-1)}.
//
// so the updates of step i-1 and the dot products of step i share one pass
// over the remaining columns.  Division by r_ii is a multiplication by the
// reciprocal, formed once per step.
//
// Reductions are deterministic: a fixed warp-shuffle tree inside a warp, a
// fixed order over warp pieces inside the CTA, then every CTA sums the G CTA
// partials in the same order.  Device-wide waits are bounded (kSpinLimitNs);
// on timeout the status word is set and every CTA returns.
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

// Plain loads that bypass L1: data written by other CTAs during this kernel.
__device__ __forceinline__ double ld_cg(const double* p) { return __ldcg(p); }

__device__ __forceinline__ double warp_sum(double v) {
  // Butterfly: every lane ends with the same value (each pairwise sum is the
  // same two operands in every lane, and + is commutative).
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic CTA-wide sum; the result is returned to every thread.
__device__ double block_sum(double v, double* s_red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) s_red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double t = lane < kWarps ? s_red[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) s_red[kWarps] = t;
  }
  __syncthreads();
  const double r = s_red[kWarps];
  __syncthreads();
  return r;
}

__device__ void set_status(int* ctl, int code, int column) {
  if (atomicCAS(&ctl[kCtlStatus], 0, code) == 0) atomicExch(&ctl[kCtlColumn], column);
}

// Device-wide barrier for a cooperative launch.  Returns false if the wait
// ran past kSpinLimitNs or another CTA already recorded a failure.
__device__ bool grid_sync(int* ctl, unsigned int& gen) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int* count = reinterpret_cast<unsigned int*>(&ctl[kCtlBarCount]);
    unsigned int* genp = reinterpret_cast<unsigned int*>(&ctl[kCtlBarGen]);
    int ok = 1;
    __threadfence();
    const unsigned int arrived = atomicAdd(count, 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(count, 0u);
      __threadfence();
      atomicExch(genp, gen + 1u);
    } else {
      const unsigned long long t0 = global_timer_ns();
      unsigned int polls = 0;
      while (ld_acquire_u32(genp) == gen) {
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
    __threadfence();
    gen += 1u;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Sum of the G per-CTA partials part[0..G), same order in every CTA.
__device__ double reduce_ctas(const double* part, int G, double* s_red) {
  if (threadIdx.x < 32) {
    double t = 0.0;
    for (int bb = threadIdx.x; bb < G; bb += 32) t += ld_cg(part + bb);
    t = warp_sum(t);
    if (threadIdx.x == 0) s_red[kWarps + 1] = t;
  }
  __syncthreads();
  const double r = s_red[kWarps + 1];
  __syncthreads();
  return r;
}

template <int V>
__global__ void __launch_bounds__(kThreads, 1) mgs_sweep_kernel(const SweepArgs a) {
  extern __shared__ __align__(16) double smem[];
  const int n = a.n;
  const int chunk = a.chunk;
  const int kmax = (n + kWarps - 1) / kWarps + 2;
  double* s_qprev = smem;                    // q_{i-1} for the chunk rows
  double* s_pprev = s_qprev + chunk;         // p_{i-1} (HP)
  double* s_pcur = s_pprev + chunk;          // p_i
  double* s_piece = s_pcur + chunk;          // kWarps x kmax warp pieces
  double* s_racc = s_piece + kWarps * kmax;  // CTA partials of the current row (relative column)
  double* s_rrow = s_racc + n;               // r_{i-1, j} during step i, then r_{i, j}
  double* s_red = s_rrow + n;                // kWarps + 2 scratch

  const int G = gridDim.x;
  const int b = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t m = a.m;
  const int64_t k0 = (int64_t)b * a.rpc;
  const int64_t k1 = (k0 + a.rpc < m) ? k0 + a.rpc : m;
  const int32_t* __restrict__ rowptr = a.rowptr;
  const int32_t* __restrict__ colidx = a.col;
  const double* __restrict__ val = a.val;
  const double* __restrict__ Z = a.Z;
  double* __restrict__ Q = a.Q;
  double* __restrict__ X = a.X;
  double* __restrict__ R = a.R;
  const int64_t ldz = a.ldz, ldq = a.ldq, ldx = a.ldx;
  const int ldr = a.ldr;
  double* part_norm = a.part + (int64_t)n * G;
  unsigned int gen = 0;

  // ---- Phase 0: R = 0; Q = Z on own rows; HP: X = A Z (one block product,
  // Algorithm 8 first line) and the partial z_1^T x_1. ----
  if (b == 0) {
    for (int64_t t = tid; t < (int64_t)n * n; t += kThreads) R[(t % n) + (t / n) * ldr] = 0.0;
  }
  if (V == kHP) {
    double s0 = 0.0;
    for (int64_t k = k0 + tid; k < k1; k += kThreads) {
      const int e0 = __ldg(rowptr + k), e1 = __ldg(rowptr + k + 1);
      for (int j0 = 0; j0 < n; j0 += 8) {
        const int w = (n - j0) < 8 ? (n - j0) : 8;
        double acc[8];
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) acc[jj] = 0.0;
        for (int e = e0; e < e1; ++e) {
          const double v = __ldg(val + e);
          const double* zc = Z + __ldg(colidx + e) + (int64_t)j0 * ldz;
#pragma unroll
          for (int jj = 0; jj < 8; ++jj)
            if (jj < w) acc[jj] = fma(v, __ldg(zc + jj * ldz), acc[jj]);
        }
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
          if (jj < w) {
            const double zk = __ldg(Z + k + (int64_t)(j0 + jj) * ldz);
            X[k + (int64_t)(j0 + jj) * ldx] = acc[jj];
            Q[k + (int64_t)(j0 + jj) * ldq] = zk;
            if (j0 + jj == 0) s0 = fma(zk, acc[0], s0);
          }
        }
      }
    }
    s0 = block_sum(s0, s_red);
    if (tid == 0) part_norm[b] = s0;
  } else {
    for (int j = 0; j < n; ++j)
      for (int64_t k = k0 + tid; k < k1; k += kThreads) Q[k + (int64_t)j * ldq] = __ldg(Z + k + (int64_t)j * ldz);
  }

  for (int i = 0; i < n; ++i) {
    // ---------------- diagonal: r_ii = sqrt(z_i^T x_i) ----------------
    if (V == kHP) {
      if (i > 0) {
        const double r = s_rrow[i];  // r_{i-1,i}
        double sl = 0.0;
        double* zi = Q + (int64_t)i * ldq;
        double* xi = X + (int64_t)i * ldx;
        const double* qp = Q + (int64_t)(i - 1) * ldq;
        const double* pp = X + (int64_t)(i - 1) * ldx;
        for (int64_t k = k0 + tid; k < k1; k += kThreads) {
          const double z = fma(-r, qp[k], zi[k]);
          const double x = fma(-r, pp[k], xi[k]);
          zi[k] = z;
          xi[k] = x;
          sl = fma(z, x, sl);
        }
        sl = block_sum(sl, s_red);
        if (tid == 0) part_norm[b] = sl;
      }
      if (!grid_sync(a.ctl, gen)) return;
    } else {
      const double* zsrc;  // column i of the working Z, complete on every row
      if (i > 0) {
        const double r = s_rrow[i];
        double* zi = Q + (int64_t)i * ldq;
        const double* qp = Q + (int64_t)(i - 1) * ldq;
        for (int64_t k = k0 + tid; k < k1; k += kThreads) zi[k] = fma(-r, qp[k], zi[k]);
        if (!grid_sync(a.ctl, gen)) return;
        zsrc = zi;
      } else {
        zsrc = Z;  // column 0 of the input equals the working column 0
      }
      // x_i = A z_i^{(i-1)}  (Algorithm 4/7: the per-column MV)
      double sl = 0.0;
      for (int64_t k = k0 + tid; k < k1; k += kThreads) {
        const int e0 = __ldg(rowptr + k), e1 = __ldg(rowptr + k + 1);
        double x = 0.0;
        for (int e = e0; e < e1; ++e) x = fma(__ldg(val + e), ld_cg(zsrc + __ldg(colidx + e)), x);
        X[k] = x;
        sl = fma(ld_cg(zsrc + k), x, sl);
      }
      sl = block_sum(sl, s_red);
      if (tid == 0) part_norm[b] = sl;
      if (!grid_sync(a.ctl, gen)) return;
    }
    const double stot = reduce_ctas(part_norm, G, s_red);
    if (!(stot > 0.0) || isinf(stot)) {
      if (b == 0 && tid == 0) set_status(a.ctl, (isnan(stot) || isinf(stot)) ? kDevNonfinite : kDevBreakdown, i + 1);
      return;  // every CTA took the same decision from the same sum
    }
    const double rii = sqrt(stot);
    const double inv = 1.0 / rii;
    if (b == 0 && tid == 0) R[i + (int64_t)i * ldr] = rii;

    if (V == kNaive) {
      // p_i = A q_i with q_i = z_i / r_ii formed on the fly (Algorithm 4's second MV).
      const double* zsrc = (i > 0) ? Q + (int64_t)i * ldq : Z;
      for (int64_t k = k0 + tid; k < k1; k += kThreads) {
        const int e0 = __ldg(rowptr + k), e1 = __ldg(rowptr + k + 1);
        double p = 0.0;
        for (int e = e0; e < e1; ++e) p = fma(__ldg(val + e), ld_cg(zsrc + __ldg(colidx + e)) * inv, p);
        X[k + ldx] = p;
      }
      // Other CTAs still gather z_i; q_i may overwrite it only after this wait.
      if (!grid_sync(a.ctl, gen)) return;
    }

    // ---------------- B pass ----------------
    const int ncols = n - 1 - i;
    for (int jr = tid; jr < ncols; jr += kThreads) s_racc[jr] = 0.0;
    double* const zi = Q + (int64_t)i * ldq;
    const double* const qprev = Q + (int64_t)(i > 0 ? i - 1 : 0) * ldq;
    const double* const pprev = (V == kHP) ? X + (int64_t)(i > 0 ? i - 1 : 0) * ldx : X;
    for (int64_t c0 = k0; c0 < k1; c0 += chunk) {
      const int crows = (int)((k1 - c0) < chunk ? (k1 - c0) : chunk);
      const int nb = (crows + 31) >> 5;
      // Stage the pivots: q_i, p_i are formed (and stored), q_{i-1}, p_{i-1} loaded.
      for (int r = tid; r < nb * 32; r += kThreads) {
        double pc = 0.0, qp = 0.0, pp = 0.0;
        if (r < crows) {
          const int64_t k = c0 + r;
          zi[k] = zi[k] * inv;  // q_i = z_i / r_ii
          if (V == kHP) {
            pc = X[k + (int64_t)i * ldx] * inv;  // p_i = x_i / r_ii (eq. (tec1))
            X[k + (int64_t)i * ldx] = pc;
          } else if (V == kHA) {
            pc = X[k] * inv;
          } else {
            pc = X[k + ldx];
          }
          if (i > 0) {
            qp = qprev[k];
            if (V == kHP) pp = pprev[k];
          }
        }
        s_pcur[r] = pc;
        s_qprev[r] = qp;
        s_pprev[r] = pp;
      }
      __syncthreads();
      const int64_t U = (int64_t)ncols * nb;  // work units: (column, 32-row block)
      if (ncols > 0) {
        int64_t u = U * warp / kWarps;
        const int64_t u1 = U * (warp + 1) / kWarps;
        const int jfirst = (int)(u / nb);
        while (u < u1) {
          const int jr = (int)(u / nb);
          const int j = i + 1 + jr;
          const int64_t uend = ((int64_t)(jr + 1) * nb < u1) ? (int64_t)(jr + 1) * nb : u1;
          const double rp = (i > 0) ? s_rrow[j] : 0.0;
          double* zc = Q + (int64_t)j * ldq + c0;
          double* xc = (V == kHP) ? X + (int64_t)j * ldx + c0 : X;
          double acc = 0.0;
          const int rbeg = (int)(u - (int64_t)jr * nb) * 32 + lane;
          int rend = (int)(uend - (int64_t)jr * nb) * 32;
          if (rend > crows) rend = crows;
          // Four rows per lane per trip: all loads are issued before the
          // arithmetic so each lane keeps several requests in flight.
          for (int r = rbeg; r < rend; r += 128) {
            double z[4], x[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int rr = r + 32 * q;
              z[q] = rr < rend ? zc[rr] : 0.0;
              x[q] = (V == kHP && i > 0 && rr < rend) ? xc[rr] : 0.0;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int rr = r + 32 * q;
              if (rr < rend) {
                if (i > 0) {
                  z[q] = fma(-rp, s_qprev[rr], z[q]);
                  zc[rr] = z[q];
                  if (V == kHP) xc[rr] = fma(-rp, s_pprev[rr], x[q]);
                }
                acc = fma(s_pcur[rr], z[q], acc);
              }
            }
          }
          acc = warp_sum(acc);
          if (lane == 0) s_piece[warp * kmax + (jr - jfirst)] = acc;
          u = uend;
        }
      }
      __syncthreads();
      // Combine the warp pieces of each column in warp order.
      for (int jr = tid; jr < ncols; jr += kThreads) {
        double t = 0.0;
        for (int w = 0; w < kWarps; ++w) {
          const int64_t w0 = U * w / kWarps, w1 = U * (w + 1) / kWarps;
          if (w0 >= w1) continue;
          const int jf = (int)(w0 / nb), jl = (int)((w1 - 1) / nb);
          if (jr >= jf && jr <= jl) t += s_piece[w * kmax + (jr - jf)];
        }
        s_racc[jr] += t;
      }
      __syncthreads();
    }
    if (ncols == 0) break;
    for (int jr = tid; jr < ncols; jr += kThreads) a.part[(int64_t)(i + 1 + jr) * G + b] = s_racc[jr];
    if (!grid_sync(a.ctl, gen)) return;
    // r_ij for j > i: the same fixed-order sum over CTAs in every CTA.
    for (int jr = warp; jr < ncols; jr += kWarps) {
      const double* pp = a.part + (int64_t)(i + 1 + jr) * G;
      double t = 0.0;
      for (int bb = lane; bb < G; bb += 32) t += ld_cg(pp + bb);
      t = warp_sum(t);
      if (lane == 0) {
        s_rrow[i + 1 + jr] = t;
        if (b == 0) R[i + (int64_t)(i + 1 + jr) * ldr] = t;
      }
    }
    __syncthreads();
  }
}

}  // namespace

static const void* sweep_fn(int variant) {
  switch (variant) {
    case kNaive: return reinterpret_cast<const void*>(mgs_sweep_kernel<kNaive>);
    case kHA: return reinterpret_cast<const void*>(mgs_sweep_kernel<kHA>);
    default: return reinterpret_cast<const void*>(mgs_sweep_kernel<kHP>);
  }
}

cudaError_t sweep_prepare(int device) {
  int optin = 0;
  cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  if (e != cudaSuccess) return e;
  for (int v = kNaive; v <= kHP; ++v) {
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, sweep_fn(v))) != cudaSuccess) return e;
    const int dyn = optin - (int)fa.sharedSizeBytes;  // static shared memory counts against the opt-in limit
    if ((e = cudaFuncSetAttribute(sweep_fn(v), cudaFuncAttributeMaxDynamicSharedMemorySize, dyn)) != cudaSuccess) return e;
  }
  return cudaSuccess;
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

cudaError_t sweep_launch(int variant, const SweepArgs& a, int grid, size_t smem, cudaStream_t s) {
  SweepArgs copy = a;
  void* args[] = {&copy};
  return cudaLaunchCooperativeKernel(sweep_fn(variant), dim3(grid), dim3(kThreads), args, smem, s);
}

}  // namespace mgsa
