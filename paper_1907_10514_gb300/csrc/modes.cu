// modes.cu -- minimisation and normal-mode Hessian of libiontrap.so (sm_103a).
//
// Minimisation (Sec. 3 "Minimisation": the equations of motion are damped to extract
// energy and the distance an ion may move in one step is limited) is damped dynamics on
// the static potential -- the pseudopotential trap of Eq. 2 (or a static RF-off trap) plus
// the Coulomb pair energy of Eq. 4.  From rest, every iteration:
//   1. a = Coulomb (the handle's pair kernel, FP32 sums in the FP32 form) + trap springs;
//      F_i = M_i a_i; stop when |F| (2-norm over all ions) < ftol
//   2. v = (v.F / F.F) F when v.F > 0, else v = 0
//   3. v += dt a; d = dt v; both scaled by s = min(1, dmax / max_i |d_i|); x += d
// Three kernels per iteration after the force evaluation; each reduction is a fixed-order
// tree per block followed by the last block folding the block partials in block order,
// so the iteration is deterministic.  No kernel waits on another.
//
// Hessian (Sec. 5 "Normal modes of motion": the mode frequencies are the eigenvalues of
// the Hessian of Eq. 4's potential): the mass-weighted second derivatives of the static
// potential, FP64, H[(3i+a)(3n) + 3j+b] = d^2V/dx_ia dx_jb / sqrt(M_i M_j), with the pair
// block k_e e^2 z_i z_j (delta_ab/r^3 - 3 r_a r_b/r^5) and the diagonal block minus the
// row's pair blocks plus M_i k_a delta_ab.
#include <algorithm>

#include "iontrap_internal.cuh"

namespace it {

struct MinState {
  double FF, vF;       // totals of the current iteration
  double scale;        // velocity projection factor v.F / F.F (0 when v.F <= 0)
  double fnorm;        // |F| of the last force evaluation
  double s;            // displacement factor of the current iteration
  long long iters;     // iterations that moved the ions
  int converged;
  unsigned cnt;        // last-block arrival counter (zero between kernels)
};

struct MinArgs {
  long long n;
  const double* coul;  // Coulomb accelerations [3][n] at x (pair kernel output)
  double* x;           // positions [3][n]
  double* v;           // velocities [3][n]
  double* a;           // accelerations [3][n] (written: trap + Coulomb at x)
  const unsigned char* sp;
  float4* hi;          // FP32 form pair stream for the next force evaluation
  float4* lo;
  double4_32a* p64;    // FP64 form pair stream
  double* part;        // block partials [blocks][2]
  MinState* st;
  double dt, dmax, ftol;
  TrapDev trap;
  SpeciesDev spc[IONTRAP_MAX_SPECIES];
};

constexpr int kMinThreads = 256;

// Set by the force kernel of an iteration and read by the later kernels of the same
// iteration only, so every block of a kernel sees the same value.  The host launches no
// more iterations than allowed.
__device__ __forceinline__ bool min_done(const MinArgs& A) { return A.st->converged != 0; }

// Fixed-order block reduction of two sums (kind 0) or of a maximum (kind 1) into v[0..1].
template <int KIND>
__device__ __forceinline__ void block_reduce2(double v[2], double* sh) {
  const int tid = threadIdx.x;
  sh[2 * tid] = v[0];
  sh[2 * tid + 1] = v[1];
  __syncthreads();
  for (int w = kMinThreads / 2; w > 0; w >>= 1) {
    if (tid < w) {
      if (KIND == 0) {
        sh[2 * tid] += sh[2 * (tid + w)];
        sh[2 * tid + 1] += sh[2 * (tid + w) + 1];
      } else {
        sh[2 * tid] = fmax(sh[2 * tid], sh[2 * (tid + w)]);
      }
    }
    __syncthreads();
  }
  v[0] = sh[0];
  v[1] = sh[1];
}

// True in the one thread of the last block to arrive (after its partial is visible).
__device__ __forceinline__ bool last_block(unsigned* cnt) {
  __shared__ unsigned s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = (atomicAdd(cnt, 1u) == gridDim.x - 1) ? 1u : 0u;
  }
  __syncthreads();
  return s_last != 0;
}

// 1: accelerations, F.F and v.F; the last block decides convergence and the projection.
__global__ void __launch_bounds__(kMinThreads) k_min_force(const __grid_constant__ MinArgs A) {
  __shared__ double sh[2 * kMinThreads];
  if (min_done(A)) return;
  const long long n = A.n;
  double acc2[2] = {0.0, 0.0};
  for (long long i = blockIdx.x * (long long)kMinThreads + threadIdx.x; i < n;
       i += (long long)gridDim.x * kMinThreads) {
    const SpeciesDev& sd = A.spc[A.sp[i]];
    double k[3];
    trap_springs(A.trap, sd, 0.0, k);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double x = A.x[c * n + i];
      const double a = A.coul[c * n + i] + (-k[c] * x);
      const double F = sd.mass * a;
      A.a[c * n + i] = a;
      acc2[0] += F * F;
      acc2[1] += A.v[c * n + i] * F;
    }
  }
  block_reduce2<0>(acc2, sh);
  if (threadIdx.x == 0) {
    A.part[2 * blockIdx.x] = acc2[0];
    A.part[2 * blockIdx.x + 1] = acc2[1];
  }
  if (last_block(&A.st->cnt) && threadIdx.x == 0) {
    double FF = 0.0, vF = 0.0;
    for (unsigned b = 0; b < gridDim.x; ++b) {
      FF += __ldcg(A.part + 2 * b);
      vF += __ldcg(A.part + 2 * b + 1);
    }
    MinState* st = A.st;
    st->FF = FF;
    st->vF = vF;
    st->fnorm = sqrt(FF);
    st->converged = st->fnorm < A.ftol;
    st->scale = vF > 0.0 ? vF / FF : 0.0;
    st->cnt = 0u;
  }
}

// 2: projected velocity plus the Euler kick; the largest displacement; the step factor
// and the iteration count.
__global__ void __launch_bounds__(kMinThreads) k_min_kick(const __grid_constant__ MinArgs A) {
  __shared__ double sh[2 * kMinThreads];
  if (min_done(A)) return;
  const long long n = A.n;
  const double scale = A.st->scale;
  double dm[2] = {0.0, 0.0};
  for (long long i = blockIdx.x * (long long)kMinThreads + threadIdx.x; i < n;
       i += (long long)gridDim.x * kMinThreads) {
    const SpeciesDev& sd = A.spc[A.sp[i]];
    double d2 = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double a = A.a[c * n + i];
      const double v = scale * (sd.mass * a) + A.dt * a;
      A.v[c * n + i] = v;
      const double d = A.dt * v;
      d2 += d * d;
    }
    dm[0] = fmax(dm[0], sqrt(d2));
  }
  block_reduce2<1>(dm, sh);
  if (threadIdx.x == 0) A.part[2 * blockIdx.x] = dm[0];
  if (last_block(&A.st->cnt) && threadIdx.x == 0) {
    double m = 0.0;
    for (unsigned b = 0; b < gridDim.x; ++b) m = fmax(m, __ldcg(A.part + 2 * b));
    A.st->s = (m > 0.0 && A.dmax < m) ? A.dmax / m : 1.0;
    A.st->iters += 1;
    A.st->cnt = 0u;
  }
}

// 3: the scaled move; the next pair-stream entries.
__global__ void __launch_bounds__(kMinThreads) k_min_move(const __grid_constant__ MinArgs A) {
  if (min_done(A)) return;
  const long long n = A.n;
  const double s = A.st->s;
  for (long long i = blockIdx.x * (long long)kMinThreads + threadIdx.x; i < n;
       i += (long long)gridDim.x * kMinThreads) {
    double xn[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double v = A.v[c * n + i];
      xn[c] = A.x[c * n + i] + s * (A.dt * v);
      A.x[c * n + i] = xn[c];
      A.v[c * n + i] = s * v;
    }
    const float w = A.spc[A.sp[i]].w;
    if (A.p64) {
      A.p64[i] = make_double4_32a(xn[0], xn[1], xn[2], (double)w);
    } else {
      float h[3], l[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        h[c] = __double2float_rn(xn[c]);
        l[c] = __double2float_rn(xn[c] - (double)h[c]);
      }
      A.hi[i] = make_float4(h[0], h[1], h[2], w);
      A.lo[i] = make_float4(l[0], l[1], l[2], 0.0f);
    }
  }
}

int min_blocks(long long n) { return (int)std::min<long long>((n + kMinThreads - 1) / kMinThreads, 1024); }

size_t min_scratch_bytes(long long n) { return sizeof(MinState) + 2 * sizeof(double) * (size_t)min_blocks(n); }

// Enqueue the three post-force kernels of one iteration.  scratch holds the MinState
// followed by the block partials.
cudaError_t launch_min_iteration(const StepArgs& s, const double* coul, void* scratch, double dt, double dmax,
                                 double ftol, int f64, int b, cudaStream_t st) {
  MinArgs A{};
  A.n = s.n;
  A.coul = coul;
  A.x = s.x;
  A.v = s.v;
  A.a = s.a;
  A.sp = s.sp;
  if (f64) {
    A.p64 = s.p64[b];
  } else {
    A.hi = s.hi[b];
    A.lo = s.lo[b];
  }
  A.st = static_cast<MinState*>(scratch);
  A.part = reinterpret_cast<double*>(static_cast<char*>(scratch) + sizeof(MinState));
  A.dt = dt;
  A.dmax = dmax;
  A.ftol = ftol;
  A.trap = s.trap;
  for (int k = 0; k < IONTRAP_MAX_SPECIES; ++k) A.spc[k] = s.spc[k];
  void* params[] = {&A};
  const dim3 grid((unsigned)min_blocks(s.n)), block(kMinThreads);
  cudaError_t e = cudaLaunchKernel((const void*)k_min_force, grid, block, params, 0, st);
  if (e == cudaSuccess) e = cudaLaunchKernel((const void*)k_min_kick, grid, block, params, 0, st);
  if (e == cudaSuccess) e = cudaLaunchKernel((const void*)k_min_move, grid, block, params, 0, st);
  return e;
}

// Progress of a minimisation, read on the host.
void min_progress(const void* host_state, long long* iters, double* fnorm, int* converged) {
  const MinState* m = static_cast<const MinState*>(host_state);
  *iters = m->iters;
  *fnorm = m->fnorm;
  *converged = m->converged;
}

size_t min_state_bytes() { return sizeof(MinState); }

// ------------------------------------------------------------------ Hessian

struct HessArgs {
  long long n;
  const double* x;
  const unsigned char* sp;
  double* H;  // [3n][3n], row-major
  double ke2;  // k_e e^2
  TrapDev trap;
  SpeciesDev spc[IONTRAP_MAX_SPECIES];
};

// Unweighted pair block d^2 (k_e e^2 z_i z_j / r) / dx_ia dx_jb for r = x_i - x_j.
__device__ __forceinline__ void pair_block(const HessArgs& A, long long i, long long j, double h[3][3]) {
  const long long n = A.n;
  double r[3], r2 = 0.0;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    r[c] = A.x[c * n + i] - A.x[c * n + j];
    r2 += r[c] * r[c];
  }
  const double rr = sqrt(r2);
  const double r3 = r2 * rr, r5 = r3 * r2;
  const double kq = A.ke2 * A.spc[A.sp[i]].z * A.spc[A.sp[j]].z;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) h[a][b] = kq * ((a == b ? 1.0 : 0.0) / r3 - 3.0 * r[a] * r[b] / r5);
}

// Off-diagonal blocks: one thread per (i, j), j along x.
__global__ void __launch_bounds__(128) k_hess_pairs(const __grid_constant__ HessArgs A) {
  const long long n = A.n;
  const long long i = blockIdx.y;
  const long long j = blockIdx.x * 128LL + threadIdx.x;
  if (j >= n || i >= n || i == j) return;
  double h[3][3];
  pair_block(A, i, j, h);
  const double w = 1.0 / sqrt(A.spc[A.sp[i]].mass * A.spc[A.sp[j]].mass);
  const long long m = 3 * n;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) A.H[(3 * i + a) * m + 3 * j + b] = h[a][b] * w;
}

// Diagonal blocks: one CTA per ion i; minus the sum over j of the pair blocks (fixed
// order tree), plus the trap springs M_i k_a, over M_i.
__global__ void __launch_bounds__(128) k_hess_diag(const __grid_constant__ HessArgs A) {
  __shared__ double sh[9][128];
  const long long n = A.n;
  const long long i = blockIdx.x;
  double acc[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) acc[q] = 0.0;
  for (long long j = threadIdx.x; j < n; j += 128) {
    if (j == i) continue;
    double h[3][3];
    pair_block(A, i, j, h);
#pragma unroll
    for (int q = 0; q < 9; ++q) acc[q] -= h[q / 3][q % 3];
  }
#pragma unroll
  for (int q = 0; q < 9; ++q) sh[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int w = 64; w > 0; w >>= 1) {
    if (threadIdx.x < w)
#pragma unroll
      for (int q = 0; q < 9; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 9) {
    const int a = threadIdx.x / 3, b = threadIdx.x % 3;
    const SpeciesDev& sd = A.spc[A.sp[i]];
    double k[3];
    trap_springs(A.trap, sd, 0.0, k);
    const double d = sh[threadIdx.x][0] + (a == b ? sd.mass * k[a] : 0.0);
    A.H[(3 * i + a) * (3 * n) + 3 * i + b] = d / sd.mass;
  }
}

cudaError_t launch_hessian(const StepArgs& s, double* d_H, cudaStream_t st) {
  HessArgs A{};
  A.n = s.n;
  A.x = s.x;
  A.sp = s.sp;
  A.H = d_H;
  A.ke2 = kE * kE / (4.0 * kPi * kEps0);
  A.trap = s.trap;
  for (int k = 0; k < IONTRAP_MAX_SPECIES; ++k) A.spc[k] = s.spc[k];
  void* params[] = {&A};
  cudaError_t e = cudaLaunchKernel((const void*)k_hess_pairs, dim3((unsigned)((s.n + 127) / 128), (unsigned)s.n),
                                   dim3(128), params, 0, st);
  if (e == cudaSuccess) e = cudaLaunchKernel((const void*)k_hess_diag, dim3((unsigned)s.n), dim3(128), params, 0, st);
  return e;
}

}  // namespace it
