// record.cu -- strided state capture and secular time averages of libiontrap.so (sm_103a).
//
// dump(filename, variables, steps) and timeAvg(variables, duration) of Sec. 3
// "Writing/reading data": every `every` steps the positions, the velocities and/or the
// velocity averaged over the last W steps are written to a device buffer.
//
// The time average needs no per-step work in the step kernels.  In kick-drift-kick
// Verlet the full-step velocity is the mean of the two half-step velocities around it,
// v_m = (v_{m-1/2} + v_{m+1/2}) / 2, and every drift moves by dt v_{m+1/2}, so
//   sum_{m=s-W+1..s} v_m = [(x_s - x_{s-W}) + (x_{s+1} - x_{s-W+1})] / (2 dt),
// with x_{m+1} = x_m + dt (v_m + dt/2 a_m) the drift the next step will make.  A snapshot
// kernel at step s - W stores x_{s-W} and x_{s-W+1}; the record kernel at step s adds
// x_s and x_{s+1}.  Both recompute the drift with the integrator's own operations.
#include <algorithm>

#include "iontrap_internal.cuh"

namespace it {

struct RecArgs {
  long long n;
  const double* x;  // state x_s, v_s, a_s [3][n]
  const double* v;
  const double* a;
  double* snap;     // [2][3][n]: x_{s-W}, x_{s-W+1}
  double* out;      // this record: fields x [3][n] blocks, in order x, v, v_avg
  double dt, hdt;
  double inv2wdt;   // 1 / (2 W dt)
  unsigned fields;
};

__global__ void __launch_bounds__(256) k_snapshot(const __grid_constant__ RecArgs A) {
  const long long n3 = 3 * A.n;
  for (long long k = blockIdx.x * 256LL + threadIdx.x; k < n3; k += (long long)gridDim.x * 256) {
    const double x = A.x[k];
    A.snap[k] = x;
    A.snap[n3 + k] = drift(x, half_kick(A.v[k], A.a[k], A.hdt), A.dt);
  }
}

__global__ void __launch_bounds__(256) k_record(const __grid_constant__ RecArgs A) {
  const long long n3 = 3 * A.n;
  for (long long k = blockIdx.x * 256LL + threadIdx.x; k < n3; k += (long long)gridDim.x * 256) {
    const double x = A.x[k], v = A.v[k];
    long long off = 0;
    if (A.fields & IONTRAP_REC_X) {
      A.out[off + k] = x;
      off += n3;
    }
    if (A.fields & IONTRAP_REC_V) {
      A.out[off + k] = v;
      off += n3;
    }
    if (A.fields & IONTRAP_REC_VAVG) {
      const double x1 = drift(x, half_kick(v, A.a[k], A.hdt), A.dt);
      A.out[off + k] = ((x - A.snap[k]) + (x1 - A.snap[n3 + k])) * A.inv2wdt;
    }
  }
}

static unsigned rec_blocks(long long n) { return (unsigned)std::min<long long>((3 * n + 255) / 256, 2048); }

cudaError_t launch_snapshot(long long n, const double* x, const double* v, const double* a, double* snap, double dt,
                            cudaStream_t st) {
  RecArgs A{};
  A.n = n, A.x = x, A.v = v, A.a = a, A.snap = snap, A.dt = dt, A.hdt = 0.5 * dt;
  void* params[] = {&A};
  return cudaLaunchKernel((const void*)k_snapshot, dim3(rec_blocks(n)), dim3(256), params, 0, st);
}

cudaError_t launch_record(long long n, const double* x, const double* v, const double* a, const double* snap,
                          double* out, unsigned fields, long long W, double dt, cudaStream_t st) {
  RecArgs A{};
  A.n = n, A.x = x, A.v = v, A.a = a, A.snap = const_cast<double*>(snap), A.out = out, A.fields = fields;
  A.dt = dt, A.hdt = 0.5 * dt, A.inv2wdt = W > 0 ? 1.0 / (2.0 * (double)W * dt) : 0.0;
  void* params[] = {&A};
  return cudaLaunchKernel((const void*)k_record, dim3(rec_blocks(n)), dim3(256), params, 0, st);
}

}  // namespace it
