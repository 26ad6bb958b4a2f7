// step_kernels.cu -- the fused timestep kernels of libiontrap.so (sm_103a).
//
// One launch = one velocity-Verlet step for one simulation (Sec. 6 "Integration"):
//   grid.x : i-blocks of T*I ions (I ions per thread, in registers)
//   grid.y : splits of the j-range, jsplit ions each, staged into shared memory by one
//            bulk TMA copy per stream (hi and lo), completing on an mbarrier
// Every CTA sums the Coulomb term (Eq. 4, direct sum, Sec. 6 "Interactions") of its
// i-block over its j-range and writes the partial to scratch.  The last CTA to finish
// an i-block (arrival counter) merges the partials in split order and runs the fused
// epilogue: trap field (Eq. 1/3) + Langevin bath (Sec. 3) + Verlet kick/drift, and
// writes the next pair stream.  The last i-block to finish advances the device step
// counter, so a chain of launches (a CUDA graph) needs no host round trip.
//
// Summation order is a function of (n, T, I, jsplit) only: j ascending inside each
// 128-wide segment (plain FP32), segments Kahan-added per CTA, CTA partials merged in
// split order.  The same configuration always gives the same bits.
#include <cstdio>

#include "iontrap_internal.cuh"

namespace it {

// ------------------------------------------------------------------ FP32 pair terms
// d = x_i - x_j from hi/lo pairs: (x_i,hi - x_j,hi) is exact for close pairs (Sterbenz)
// and the lo difference restores the bits FP32 rounding dropped from both positions.
template <int I, bool DIAG>
__device__ __forceinline__ void segment_f32(const float4* __restrict__ sh, const float4* __restrict__ sl, int g0,
                                            int g1, long long jbase, const float (&xh)[I][3],
                                            const float (&xl)[I][3], const long long (&ii)[I],
                                            float (&acc)[I][3]) {
#pragma unroll 4
  for (int j = g0; j < g1; ++j) {
    const float4 ph = sh[j];
    const float4 pl = sl[j];
#pragma unroll
    for (int k = 0; k < I; ++k) {
      const float dx = (xh[k][0] - ph.x) + (xl[k][0] - pl.x);
      const float dy = (xh[k][1] - ph.y) + (xl[k][1] - pl.y);
      const float dz = (xh[k][2] - ph.z) + (xl[k][2] - pl.z);
      const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
      float ri = rsqrt_approx(r2);
      if (DIAG) ri = (jbase + j == ii[k]) ? 0.0f : ri;
      const float ri2 = ri * ri;
      const float s = (ph.w * ri) * ri2;  // z_j / r^3
      acc[k][0] = fmaf(s, dx, acc[k][0]);
      acc[k][1] = fmaf(s, dy, acc[k][1]);
      acc[k][2] = fmaf(s, dz, acc[k][2]);
    }
  }
}

template <int I, bool DIAG>
__device__ __forceinline__ void segment_f64(const double4* __restrict__ sp, int g0, int g1, long long jbase,
                                            const double (&xi)[I][3], const long long (&ii)[I],
                                            double (&acc)[I][3]) {
#pragma unroll 2
  for (int j = g0; j < g1; ++j) {
    const double4 p = sp[j];
#pragma unroll
    for (int k = 0; k < I; ++k) {
      const double dx = xi[k][0] - p.x;
      const double dy = xi[k][1] - p.y;
      const double dz = xi[k][2] - p.z;
      const double r2 = dx * dx + dy * dy + dz * dz;
      double ri = rsqrt(r2);
      if (DIAG) ri = (jbase + j == ii[k]) ? 0.0 : ri;
      const double s = p.w * ri * ri * ri;
      acc[k][0] += s * dx;
      acc[k][1] += s * dy;
      acc[k][2] += s * dz;
    }
  }
}

// Stage the CTA's j-range (bytes per stream) with bulk TMA; every thread waits with a
// time limit.  Returns false (error flag set, copies drained) if the wait expired.
__device__ __forceinline__ bool stage_jrange(uint64_t* bar, void* d0, const void* s0, void* d1, const void* s1,
                                             uint32_t bytes, int* err) {
  if (threadIdx.x == 0) mbar_init(bar, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_arrive_expect_tx(bar, s1 ? 2u * bytes : bytes);
    tma_bulk_g2s(d0, s0, bytes, bar);
    if (s1) tma_bulk_g2s(d1, s1, bytes, bar);
  }
  const bool ok = mbar_wait_bounded(bar, 0, kWaitLimitNs);
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) {
      atomicOr(err, ERR_TIMEOUT);
      mbar_wait_bounded(bar, 0, kWaitLimitNs);
    }
    __syncthreads();
    return false;
  }
  return true;
}

// Arrival at the i-block counter; true in the last CTA of the i-block.
__device__ __forceinline__ bool arrive_last(unsigned* cnt, unsigned expected, int* s_flag) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(cnt, 1u);
    *s_flag = (prev == expected - 1u);
  }
  __syncthreads();
  const bool last = *s_flag != 0;
  if (last) __threadfence();
  return last;
}

// Reset the i-block counter and, in the last i-block, advance the step counter.
__device__ __forceinline__ void finish_iblock(const StepArgs& A, long long ns) {
  __syncthreads();
  if (threadIdx.x == 0) {
    A.cnt[blockIdx.x] = 0u;
    __threadfence();
    const unsigned prev = atomicAdd(A.done, 1u);
    if (prev == gridDim.x - 1u) {
      *A.done = 0u;
      if (A.mode == MODE_STEP) *A.step = ns + 1;
      __threadfence();
    }
  }
}

__device__ __forceinline__ double force_time_cos(const StepArgs& A, long long ns) {
  const long long nf = (A.mode == MODE_STEP) ? ns + 1 : ns;
  if (A.trap.flags & (IONTRAP_RF_OFF | IONTRAP_TRAP_OFF)) return 0.0;
  return cos(A.trap.Omega * ((double)nf * A.trap.dt));
}

// ------------------------------------------------------------------ FP32 form
template <int T, int I>
__global__ void __launch_bounds__(T) k_step_f32(const __grid_constant__ StepArgs A) {
  extern __shared__ __align__(128) unsigned char smraw[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ int s_flag;
  __shared__ double s_cos;
  float4* sh = reinterpret_cast<float4*>(smraw);
  float4* sl = sh + A.jsplit;

  const int tid = threadIdx.x;
  const long long n = A.n;
  const long long i0 = (long long)blockIdx.x * (T * I);
  const long long j0 = (long long)blockIdx.y * A.jsplit;
  const int jn = (int)min((long long)A.jsplit, n - j0);
  const long long ns = *A.step;
  const int rb = (A.mode == MODE_STEP) ? (int)((ns + 1) & 1) : (int)(ns & 1);
  const bool coulomb = !(A.trap.flags & IONTRAP_COULOMB_OFF);

  float ks[I][3], kc[I][3];
#pragma unroll
  for (int k = 0; k < I; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c) ks[k][c] = kc[k][c] = 0.0f;

  if (coulomb) {
    if (!stage_jrange(&bar, sh, A.hi[rb] + j0, sl, A.lo[rb] + j0, (uint32_t)jn * 16u, A.err)) return;
    float xh[I][3], xl[I][3];
    long long ii[I];
#pragma unroll
    for (int k = 0; k < I; ++k) {
      ii[k] = i0 + k * T + tid;
      float4 h = make_float4(0.f, 0.f, 0.f, 0.f), l = h;
      if (ii[k] < n) {
        h = A.hi[rb][ii[k]];
        l = A.lo[rb][ii[k]];
      }
      xh[k][0] = h.x, xh[k][1] = h.y, xh[k][2] = h.z;
      xl[k][0] = l.x, xl[k][1] = l.y, xl[k][2] = l.z;
    }
    const long long iend = i0 + T * I;
    for (int g0 = 0; g0 < jn; g0 += kSeg) {
      const int g1 = min(g0 + kSeg, jn);
      float acc[I][3];
#pragma unroll
      for (int k = 0; k < I; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[k][c] = 0.0f;
      const bool diag = (j0 + g0 < iend) && (i0 < j0 + g1);
      if (diag)
        segment_f32<I, true>(sh, sl, g0, g1, j0, xh, xl, ii, acc);
      else
        segment_f32<I, false>(sh, sl, g0, g1, j0, xh, xl, ii, acc);
      // Kahan: value = ks - kc
#pragma unroll
      for (int k = 0; k < I; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float y = acc[k][c] - kc[k][c];
          const float t = ks[k][c] + y;
          kc[k][c] = (t - ks[k][c]) - y;
          ks[k][c] = t;
        }
    }
  }

  // partials: part[((split*3 + c)*2 + {0: sum, 1: compensation}) * n + i]
  float* part = reinterpret_cast<float*>(A.part);
#pragma unroll
  for (int k = 0; k < I; ++k) {
    const long long i = i0 + k * T + tid;
    if (i < n) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        __stcg(part + ((blockIdx.y * 3ll + c) * 2 + 0) * n + i, ks[k][c]);
        __stcg(part + ((blockIdx.y * 3ll + c) * 2 + 1) * n + i, kc[k][c]);
      }
    }
  }
  if (!arrive_last(&A.cnt[blockIdx.x], gridDim.y, &s_flag)) return;

  if (tid == 0) s_cos = force_time_cos(A, ns);
  __syncthreads();
  const double cosv = s_cos;
  const int wb = rb ^ 1;
  const int nsplit = gridDim.y;
#pragma unroll
  for (int k = 0; k < I; ++k) {
    const long long i = i0 + k * T + tid;
    if (i >= n) continue;
    double S[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float s = 0.0f, cc = 0.0f;
      for (int p = 0; p < nsplit; ++p) {
        const float ps = __ldcg(part + ((p * 3ll + c) * 2 + 0) * n + i);
        const float pc = __ldcg(part + ((p * 3ll + c) * 2 + 1) * n + i);
        const float y = ps - cc;
        const float t = s + y;
        cc = ((t - s) - y) + pc;
        s = t;
      }
      S[c] = (double)s - (double)cc;
    }
    epilogue_ion<false>(A, i, S, cosv, ns, wb);
  }
  finish_iblock(A, ns);
}

// ------------------------------------------------------------------ FP64 plain form
template <int T, int I>
__global__ void __launch_bounds__(T) k_step_f64(const __grid_constant__ StepArgs A) {
  extern __shared__ __align__(128) unsigned char smraw[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ int s_flag;
  __shared__ double s_cos;
  double4* sp = reinterpret_cast<double4*>(smraw);

  const int tid = threadIdx.x;
  const long long n = A.n;
  const long long i0 = (long long)blockIdx.x * (T * I);
  const long long j0 = (long long)blockIdx.y * A.jsplit;
  const int jn = (int)min((long long)A.jsplit, n - j0);
  const long long ns = *A.step;
  const int rb = (A.mode == MODE_STEP) ? (int)((ns + 1) & 1) : (int)(ns & 1);
  const bool coulomb = !(A.trap.flags & IONTRAP_COULOMB_OFF);

  double acc[I][3];
#pragma unroll
  for (int k = 0; k < I; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[k][c] = 0.0;

  if (coulomb) {
    if (!stage_jrange(&bar, sp, A.p64[rb] + j0, nullptr, nullptr, (uint32_t)jn * 32u, A.err)) return;
    double xi[I][3];
    long long ii[I];
#pragma unroll
    for (int k = 0; k < I; ++k) {
      ii[k] = i0 + k * T + tid;
      double4 p = make_double4(0., 0., 0., 0.);
      if (ii[k] < n) p = A.p64[rb][ii[k]];
      xi[k][0] = p.x, xi[k][1] = p.y, xi[k][2] = p.z;
    }
    const long long iend = i0 + T * I;
    for (int g0 = 0; g0 < jn; g0 += kSeg) {
      const int g1 = min(g0 + kSeg, jn);
      const bool diag = (j0 + g0 < iend) && (i0 < j0 + g1);
      if (diag)
        segment_f64<I, true>(sp, g0, g1, j0, xi, ii, acc);
      else
        segment_f64<I, false>(sp, g0, g1, j0, xi, ii, acc);
    }
  }

  double* part = reinterpret_cast<double*>(A.part);
#pragma unroll
  for (int k = 0; k < I; ++k) {
    const long long i = i0 + k * T + tid;
    if (i < n) {
#pragma unroll
      for (int c = 0; c < 3; ++c) __stcg(part + (blockIdx.y * 3ll + c) * n + i, acc[k][c]);
    }
  }
  if (!arrive_last(&A.cnt[blockIdx.x], gridDim.y, &s_flag)) return;

  if (tid == 0) s_cos = force_time_cos(A, ns);
  __syncthreads();
  const double cosv = s_cos;
  const int wb = rb ^ 1;
  const int nsplit = gridDim.y;
#pragma unroll
  for (int k = 0; k < I; ++k) {
    const long long i = i0 + k * T + tid;
    if (i >= n) continue;
    double S[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      double s = 0.0;
      for (int p = 0; p < nsplit; ++p) s += __ldcg(part + (p * 3ll + c) * n + i);
      S[c] = s;
    }
    epilogue_ion<true>(A, i, S, cosv, ns, wb);
  }
  finish_iblock(A, ns);
}

// ------------------------------------------------------------------ helpers
// Write pair stream b from the FP64 positions x_n (create and force evaluation).
__global__ void k_prep(const __grid_constant__ StepArgs A, int b, int f64) {
  const long long n = A.n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double xn[3] = {A.x[i], A.x[n + i], A.x[2 * n + i]};
    const float w = A.spc[A.sp[i]].w;
    if (f64)
      write_pair<true>(A, b, i, xn, w);
    else
      write_pair<false>(A, b, i, xn, w);
  }
}

// Write pair stream b from a full state (x_n, v_n, a_n): the drifted positions
// x_{n+1} = x_n + dt (v_n + dt/2 a_n), by the same operations the epilogue uses.
__global__ void k_restore(const __grid_constant__ StepArgs A, int b, int f64) {
  const long long n = A.n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double xn[3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
      xn[c] = drift(A.x[c * n + i], half_kick(A.v[c * n + i], A.a[c * n + i], A.trap.hdt), A.trap.dt);
    const float w = A.spc[A.sp[i]].w;
    if (f64)
      write_pair<true>(A, b, i, xn, w);
    else
      write_pair<false>(A, b, i, xn, w);
  }
}

__global__ void k_normals(unsigned long long seed, long long counter, const long long* ids, long long m, int f64,
                          double* z) {
  const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= m) return;
  double t[3];
  if (f64)
    normals3_f64(seed, counter, ids[k], t);
  else
    normals3_f32(seed, counter, ids[k], t);
  z[k] = t[0];
  z[m + k] = t[1];
  z[2 * m + k] = t[2];
}

// ------------------------------------------------------------------ registry
struct KernelEntry {
  int f64, T, I;
  const void* fn;
};

static const KernelEntry kKernels[] = {
    {0, 64, 1, (const void*)k_step_f32<64, 1>},    {0, 64, 2, (const void*)k_step_f32<64, 2>},
    {0, 64, 4, (const void*)k_step_f32<64, 4>},    {0, 128, 1, (const void*)k_step_f32<128, 1>},
    {0, 128, 2, (const void*)k_step_f32<128, 2>},  {0, 128, 4, (const void*)k_step_f32<128, 4>},
    {0, 256, 1, (const void*)k_step_f32<256, 1>},  {0, 256, 2, (const void*)k_step_f32<256, 2>},
    {0, 256, 4, (const void*)k_step_f32<256, 4>},  {1, 64, 1, (const void*)k_step_f64<64, 1>},
    {1, 128, 1, (const void*)k_step_f64<128, 1>},  {1, 128, 2, (const void*)k_step_f64<128, 2>},
    {1, 256, 1, (const void*)k_step_f64<256, 1>},
};

const void* step_kernel(int f64, int T, int I) {
  for (const auto& e : kKernels)
    if (e.f64 == f64 && e.T == T && e.I == I) return e.fn;
  return nullptr;
}

const void* prep_kernel() { return (const void*)k_prep; }
const void* restore_kernel() { return (const void*)k_restore; }

cudaError_t launch_normals(unsigned long long seed, long long counter, const long long* d_ids, long long m,
                           int f64, double* d_z, cudaStream_t st) {
  const int T = 128;
  const long long blocks = (m + T - 1) / T;
  k_normals<<<(unsigned)blocks, T, 0, st>>>(seed, counter, d_ids, m, f64, d_z);
  return cudaGetLastError();
}

}  // namespace it
