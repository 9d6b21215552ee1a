// Set-up, point-operator, probe-generation and reduction kernels.
#include <cuda_bf16.h>

#include <algorithm>

#include "tp_internal.h"

namespace tp {

namespace {

constexpr int RED_THREADS = 256;

// c2 = dt^2 v^2 / h^2 formed in fp64 and rounded once: an fp32 product chain
// is off by a few ulp, i.e. a velocity error of ~1e-7 whose phase error grows
// linearly with time (the dominant fp32 trace error after thousands of steps).
__global__ void prep_c2_kernel(Layout L, const float* __restrict__ vel, double coef, float* __restrict__ c2) {
  const long long n = (long long)L.nx * L.ny * L.nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double v = vel[i];
    c2[L.off_flat(i)] = (float)(coef * v * v);
  }
}

__global__ void vmax_kernel(const float* __restrict__ vel, long long n, unsigned int* out) {
  float m = 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf(vel[i]));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));  // non-negative floats order as integers
}

__global__ void prep_points_kernel(Layout L, Weights W, const int64_t* __restrict__ idx, long long n,
                                   const float* __restrict__ vel, double dt2, long long* __restrict__ off,
                                   float* __restrict__ cinj, int* err) {
  const long long N = (long long)L.nx * L.ny * L.nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long p = idx[i];
    if (p < 0 || p >= N) {  // reject: the point operators skip negative offsets
      off[i] = -1;
      cinj[i] = 0.f;
      atomicOr(err, 2);
    } else {
      off[i] = L.off_flat(p);
      const double v = vel[p];
      // inside the absorbing layer the injected value is divided by 1 + a like the step
      const long long x = p % L.nx, y = (p / L.nx) % L.ny, z = p / ((long long)L.nx * L.ny);
      const double a = (double)sponge_a(L, W, z, y, x);
      cinj[i] = (float)(dt2 * v * v / (1.0 + a));
    }
  }
}

__device__ __forceinline__ void inject_one(const PointArgs& a, int s, int k) {
  const long long k2 = (long long)s * a.ninj + k;
  const long long o = a.inj_off[k2];
  if (o < 0) return;
  const float v = a.inj_coef[k2] * a.inj_val[s * a.inj_val_ss + k];
  float* f = a.field_inj + s * a.inj_ss + o;
  *f = *f + v;
  if (a.field_inj2) {
    float* f2 = a.field_inj2 + s * a.inj2_ss + o;
    *f2 = *f2 + v;
  }
}

// Sampling threads, then one thread per injection entry that is alone at its
// node, then one thread per shot that adds the entries sharing nodes, in
// index order: every node's sum has a fixed order (deterministic results).
__global__ void point_kernel(PointArgs a) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long ns = (long long)a.nshots * a.nsamp;
  if (i < ns) {
    const int s = (int)(i / a.nsamp), j = (int)(i % a.nsamp);
    const long long o = a.samp_off[i];
    const float v = o >= 0 ? a.field_samp[s * a.samp_ss + o] : 0.f;
    if (a.samp_out) a.samp_out[s * a.samp_out_ss + j] = v;
    if (a.acc) a.acc[i] += (double)v * (double)a.acc_val[s * a.acc_val_ss + j];
    return;
  }
  const long long k2 = i - ns;
  const long long ni = (long long)a.nshots * a.ninj;
  if (k2 < ni) {
    if (a.inj_alone[k2]) inject_one(a, (int)(k2 / a.ninj), (int)(k2 % a.ninj));
    return;
  }
  const long long s = k2 - ni;
  if (a.ninj > 0 && s < a.nshots) {
    const int nd = a.inj_nshared[s];
    for (int d = 0; d < nd; ++d) inject_one(a, (int)s, a.inj_shared[s * a.ninj + d]);
  }
}

// Nodes with more than one entry of a point set (counts over the padded
// field of each shot; `cnt` is zero on entry)
__global__ void point_count_kernel(const long long* __restrict__ off, long long n, int per_shot, long long field,
                                   int* cnt) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const long long o = off[k];
    if (o >= 0) atomicAdd(cnt + (k / per_shot) * field + o, 1);
  }
}

// One block per shot: alone[k] for every entry, and the entries whose node
// has several, compacted in index order into shared[shot][..], nshared[shot]
__global__ void __launch_bounds__(256) point_group_kernel(const long long* __restrict__ off, int per_shot,
                                                          long long field, const int* __restrict__ cnt,
                                                          unsigned char* alone, int* shared, int* nshared) {
  __shared__ int warp_cnt[8];
  __shared__ int base_cnt;
  const int s = blockIdx.x, tid = threadIdx.x;
  if (tid == 0) base_cnt = 0;
  __syncthreads();
  for (int b = 0; b < per_shot; b += 256) {
    const int k = b + tid;
    bool dup = false;
    if (k < per_shot) {
      const long long o = off[(long long)s * per_shot + k];
      const bool one = o < 0 || cnt[(long long)s * field + o] == 1;
      alone[(long long)s * per_shot + k] = one ? 1 : 0;
      dup = !one;
    }
    const unsigned m = __ballot_sync(0xffffffffu, dup);
    if ((tid & 31) == 0) warp_cnt[tid >> 5] = __popc(m);
    __syncthreads();
    int before = base_cnt;
    for (int w = 0; w < (tid >> 5); ++w) before += warp_cnt[w];
    if (dup) shared[(long long)s * per_shot + before + __popc(m & ((1u << (tid & 31)) - 1u))] = k;
    __syncthreads();
    if (tid == 0)
      for (int w = 0; w < 8; ++w) base_cnt += warp_cnt[w];
    __syncthreads();
  }
  if (tid == 0) nshared[s] = base_cnt;
}

// SplitMix64 (Steele, Lea & Flood 2014): the n-th output of a generator whose
// state starts at s is mix(s + n * 0x9E3779B97F4A7C15).
__device__ __forceinline__ uint64_t sm64(uint64_t s, uint64_t n) {
  uint64_t z = s + n * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// Probe entry Z[t][i] of shot `shot`: key chain seed -> shot -> column, then
// draws indexed by time.  Rademacher: sign of the top bit of one draw.
// Gaussian: Irwin-Hall sum of the high 32 bits of 12 draws, centred, floored
// to a multiple of 2^12 and mapped to the odd multiple (2k+1) 2^-21 (exact in
// fp32).  Identity: Z = I.  User: copy.
__global__ void probes_kernel(int kind, int nt, int r, uint64_t seed, int shot0, int nshots,
                              const float* __restrict__ Zu, float* __restrict__ Q) {
  const long long n = (long long)nshots * nt * r;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(e / ((long long)nt * r));
    const long long rem = e % ((long long)nt * r);
    const int t = (int)(rem / r), i = (int)(rem % r);
    float z;
    if (kind == 2) {
      z = (t == i) ? 1.f : 0.f;
    } else if (kind == 3) {
      z = Zu[e];
    } else {
      const uint64_t ks = sm64(seed, (uint64_t)(shot0 + s) + 1);
      const uint64_t kc = sm64(ks, (uint64_t)i + 1);
      if (kind == 0) {
        z = (sm64(kc, (uint64_t)t + 1) >> 63) ? -1.f : 1.f;
      } else {
        long long S = 0;
#pragma unroll
        for (int d = 0; d < 12; ++d) S += (long long)(sm64(kc, 12ULL * (uint64_t)t + d + 1) >> 32);
        S -= 6LL << 32;
        const long long fl = S >= 0 ? (S >> 12) : -((-S + 4095) >> 12);
        z = (float)(2 * fl + 1) * 4.76837158203125e-07f;  // 2^-21
      }
    }
    Q[e] = z;
  }
}

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[RED_THREADS / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < RED_THREADS / 32 ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  __syncthreads();
  return t;
}

// res = d - dobs (in place), part[block] = sum res^2 over a fixed grid-stride set
__global__ void __launch_bounds__(RED_THREADS) residual_kernel(float* __restrict__ d, const float* __restrict__ dobs,
                                                                long long n, double* __restrict__ part) {
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float r = d[i] - dobs[i];
    d[i] = r;
    acc += (double)r * (double)r;
  }
  const double t = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void __launch_bounds__(RED_THREADS) sumsq_kernel(const float* __restrict__ a, long long n,
                                                             double* __restrict__ part) {
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    acc += (double)a[i] * (double)a[i];
  const double t = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void __launch_bounds__(RED_THREADS) finalize_kernel(const double* __restrict__ part, int nblk,
                                                                double scale, double* out, int do_sqrt,
                                                                const int* err) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) acc += part[i];
  const double t = block_sum(acc);
  if (threadIdx.x == 0) {
    double v = do_sqrt ? sqrt(t) * scale : t * scale;
    if (err && (*err & 1)) v = __longlong_as_double(0x7ff8000000000000LL);  // NaN on a timed-out wait
    *out = v;
  }
}

// grad[x] = -scale_h2 * vel[x]^2 * sum_s gacc[s][off(x)]
__global__ void finish_grad_kernel(Layout L, const float* __restrict__ vel, const float* __restrict__ gacc,
                                   int nshots, long long gacc_ss, float scale_h2, float* __restrict__ grad,
                                   int times_v2) {
  const long long n = (long long)L.nx * L.ny * L.nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long o = L.off_flat(i);
    float acc = 0.f;
    for (int s = 0; s < nshots; ++s) acc += gacc[s * gacc_ss + o];
    const float v = times_v2 ? vel[i] : 1.0f;
    grad[i] = -scale_h2 * v * v * acc;
  }
}

__global__ void source_into_acc_kernel(const long long* __restrict__ soff, const int64_t* __restrict__ src,
                                       const float* __restrict__ vel, double dt2, const float* __restrict__ qbar,
                                       int nsrc, int nshots, int r, float* __restrict__ U, long long u_ss,
                                       long long field) {
  const int i = threadIdx.x;  // one thread per probe column, shots and sources in a fixed order
  if (i >= r || blockIdx.x != 0) return;
  for (int s = 0; s < nshots; ++s)
    for (int k = 0; k < nsrc; ++k) {
      const long long o = soff[(long long)s * nsrc + k];
      if (o < 0) continue;
      const double v = vel[src[(long long)s * nsrc + k]];
      const float coef = (float)(dt2 * v * v);  // dt^2 v^2, undamped: the factor of S^T qbar in ubar
      U[s * u_ss + (long long)i * field + o] += coef * qbar[((long long)s * nsrc + k) * r + i];
    }
}

__global__ void qbar_kernel(const float* __restrict__ Q, int nt, int r, const float* __restrict__ wav, int nsrc,
                            int nshots, int jlo, int jhi, int qshift, float* __restrict__ qbar) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nshots * nsrc * r) return;
  const int s = e / (nsrc * r), k = (e / r) % nsrc, i = e % r;
  double acc = 0.0;
  for (int j = jlo; j <= jhi; ++j)
    acc += (double)Q[((long long)s * nt + j + qshift) * r + i] * (double)wav[((long long)s * nt + j) * nsrc + k];
  qbar[e] = (float)acc;
}

// value of accumulator i at element o of one shot's accumulator block
__device__ __forceinline__ float acc_value(const void* P, int acc, int r, int i, long long field, long long o) {
  if (acc == 0) return static_cast<const float*>(P)[(long long)i * field + o];
  const __nv_bfloat16* h = static_cast<const __nv_bfloat16*>(P);
  float v = __bfloat162float(h[(long long)i * field + o]);
  if (acc == 2) v += __bfloat162float(h[(long long)(r + i) * field + o]);
  return v;
}

__global__ void acc_to_f32_kernel(const void* __restrict__ P, int acc, int r, int i, long long field, int nshots,
                                  float* __restrict__ out, long long out_ss) {
  const long long per = acc == 2 ? 2LL * r * field : (long long)r * field;  // elements per shot
  const long long n = (long long)nshots * field;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(e / field);
    const long long o = e % field;
    const void* Ps = acc == 0 ? (const void*)(static_cast<const float*>(P) + s * per)
                              : (const void*)(static_cast<const __nv_bfloat16*>(P) + s * per);
    out[s * out_ss + o] = acc_value(Ps, acc, r, i, field, o);
  }
}

__global__ void chain_velocity_kernel(const float* __restrict__ vel, float* __restrict__ grad, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float v = vel[i];
    grad[i] *= -2.0f / (v * v * v);
  }
}

__global__ void source_term_kernel(Layout L, const float* __restrict__ vel, const int64_t* __restrict__ src,
                                   const long long* __restrict__ soff, int nsrc, int nshots, float scale,
                                   const float* __restrict__ qbar, const void* __restrict__ V, int acc_mode, int r,
                                   long long v_ss, const double* __restrict__ srcacc, float* grad) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  const long long N = (long long)L.nx * L.ny * L.nz;
  for (int s = 0; s < nshots; ++s)
    for (int k = 0; k < nsrc; ++k) {
      const long long p = src[(long long)s * nsrc + k];
      const long long o = soff[(long long)s * nsrc + k];
      if (p < 0 || p >= N || o < 0) continue;
      double acc = 0.0;
      if (srcacc) {
        acc = srcacc[(long long)s * nsrc + k];
      } else {
        const void* Vs = acc_mode == 0 ? (const void*)(static_cast<const float*>(V) + s * v_ss)
                                       : (const void*)(static_cast<const __nv_bfloat16*>(V) + s * v_ss);
        for (int i = 0; i < r; ++i)
          acc += (double)qbar[((long long)s * nsrc + k) * r + i] * (double)acc_value(Vs, acc_mode, r, i, L.field, o);
      }
      const float v = vel[p];
      grad[p] += (float)(-(double)scale * (double)v * (double)v * acc);
    }
}

int grid_for(long long n, int threads, int cap = 8192) {
  return (int)std::max<long long>(1, std::min<long long>((n + threads - 1) / threads, cap));
}

}  // namespace

cudaError_t launch_prep_c2(const Layout& L, const float* vel, double coef, float* c2, cudaStream_t s) {
  prof_before(5, s);
  const long long n = (long long)L.nx * L.ny * L.nz;
  prep_c2_kernel<<<grid_for(n, 256), 256, 0, s>>>(L, vel, coef, c2);
  prof_after(5, s);
  return cudaGetLastError();
}

cudaError_t launch_vmax(const float* vel, long long n, unsigned int* out, cudaStream_t s) {
  prof_before(5, s);
  vmax_kernel<<<grid_for(n, 256, 2048), 256, 0, s>>>(vel, n, out);
  prof_after(5, s);
  return cudaGetLastError();
}

cudaError_t launch_prep_points(const Layout& L, const Weights& W, const int64_t* idx, long long n, const float* vel,
                               double dt2, long long* off, float* cinj, int* err, cudaStream_t s) {
  prof_before(5, s);
  prep_points_kernel<<<grid_for(n, 256), 256, 0, s>>>(L, W, idx, n, vel, dt2, off, cinj, err);
  prof_after(5, s);
  return cudaGetLastError();
}

cudaError_t launch_point_groups(const long long* off, int per_shot, int nshots, long long field, int* cnt_scratch,
                                unsigned char* alone, int* shared, int* nshared, cudaStream_t s) {
  prof_before(5, s);
  cudaError_t e = cudaMemsetAsync(cnt_scratch, 0, (size_t)nshots * field * sizeof(int), s);
  if (e == cudaSuccess) {
    const long long n = (long long)nshots * per_shot;
    point_count_kernel<<<grid_for(n, 256), 256, 0, s>>>(off, n, per_shot, field, cnt_scratch);
    point_group_kernel<<<nshots, 256, 0, s>>>(off, per_shot, field, cnt_scratch, alone, shared, nshared);
    e = cudaGetLastError();
  }
  prof_after(5, s);
  return e;
}

cudaError_t launch_point(const PointArgs& a, cudaStream_t s) {
  const long long n = (long long)a.nshots * (a.nsamp + a.ninj) + (a.ninj > 0 ? a.nshots : 0);
  if (n == 0) return cudaSuccess;
  prof_before(3, s);
  point_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a);
  prof_after(3, s);
  return cudaGetLastError();
}

cudaError_t launch_probes(int kind, int nt, int r, uint64_t seed, int shot0, int nshots, const float* Z_user,
                          float* Q, cudaStream_t s) {
  prof_before(5, s);
  const long long n = (long long)nshots * nt * r;
  probes_kernel<<<grid_for(n, 256), 256, 0, s>>>(kind, nt, r, seed, shot0, nshots, Z_user, Q);
  prof_after(5, s);
  return cudaGetLastError();
}

cudaError_t launch_residual(float* d, const float* dobs, long long n, double* part, int nblk, cudaStream_t s) {
  prof_before(4, s);
  residual_kernel<<<nblk, RED_THREADS, 0, s>>>(d, dobs, n, part);
  prof_after(4, s);
  return cudaGetLastError();
}

cudaError_t launch_sumsq(const float* a, long long n, double* part, int nblk, cudaStream_t s) {
  prof_before(4, s);
  sumsq_kernel<<<nblk, RED_THREADS, 0, s>>>(a, n, part);
  prof_after(4, s);
  return cudaGetLastError();
}

cudaError_t launch_finalize_sum(const double* part, int nblk, double scale, double* out, int sqrt_result,
                                const int* err, cudaStream_t s) {
  prof_before(4, s);
  finalize_kernel<<<1, RED_THREADS, 0, s>>>(part, nblk, scale, out, sqrt_result, err);
  prof_after(4, s);
  return cudaGetLastError();
}

cudaError_t launch_source_into_acc(const long long* src_off, const int64_t* src, const float* vel, double dt2,
                                   const float* qbar, int nsrc,
                                   int nshots, int r, float* U, long long u_ss, long long field, cudaStream_t s) {
  prof_before(5, s);
  source_into_acc_kernel<<<1, 64, 0, s>>>(src_off, src, vel, dt2, qbar, nsrc, nshots, r, U, u_ss, field);
  prof_after(5, s);
  return cudaGetLastError();
}

cudaError_t launch_finish_grad(const Layout& L, const float* vel, const float* gacc, int nshots, long long gacc_ss,
                               float scale_h2, float* grad, cudaStream_t s, int times_v2) {
  prof_before(5, s);
  const long long n = (long long)L.nx * L.ny * L.nz;
  finish_grad_kernel<<<grid_for(n, 256), 256, 0, s>>>(L, vel, gacc, nshots, gacc_ss, scale_h2, grad, times_v2);
  prof_after(5, s);
  return cudaGetLastError();
}

cudaError_t launch_qbar(const float* Q, int nt, int r, const float* wav, int nsrc, int nshots, int jlo, int jhi,
                        int qshift, float* qbar, cudaStream_t s) {
  prof_before(5, s);
  const int n = nshots * nsrc * r;
  qbar_kernel<<<(n + 127) / 128, 128, 0, s>>>(Q, nt, r, wav, nsrc, nshots, jlo, jhi, qshift, qbar);
  prof_after(5, s);
  return cudaGetLastError();
}

cudaError_t launch_source_term(const Layout& L, const float* vel, const int64_t* src_dense, const long long* src_off,
                               int nsrc, int nshots, float scale, const float* qbar, const void* V, int acc, int r,
                               long long v_ss, const double* srcacc, float* grad, cudaStream_t s) {
  prof_before(5, s);
  source_term_kernel<<<1, 32, 0, s>>>(L, vel, src_dense, src_off, nsrc, nshots, scale, qbar, V, acc, r, v_ss, srcacc,
                                      grad);
  prof_after(5, s);
  return cudaGetLastError();
}

cudaError_t launch_acc_to_f32(const void* P, int acc, int r, int i, long long field, int nshots, float* out,
                              long long out_ss, cudaStream_t s) {
  prof_before(5, s);
  acc_to_f32_kernel<<<grid_for((long long)nshots * field, 256), 256, 0, s>>>(P, acc, r, i, field, nshots, out, out_ss);
  prof_after(5, s);
  return cudaGetLastError();
}

cudaError_t launch_chain_velocity(const float* vel, float* grad, long long n, cudaStream_t s) {
  prof_before(5, s);
  chain_velocity_kernel<<<grid_for(n, 256), 256, 0, s>>>(vel, grad, n);
  prof_after(5, s);
  return cudaGetLastError();
}

}  // namespace tp
