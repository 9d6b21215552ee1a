// Range-finding probes (Eq. 6): Q_s = qr(D_s D_s^T Z_s) for every shot s,
// D_s the observed record as an nt x nrec matrix and Z_s random probes.
//
//   W = D^T Z   (nrec x r)   one thread per receiver, fp64 accumulation
//   Y = D W     (nt x r)     one warp per time level, fp64, warp reduction
//   Q = orth(Y)              classical Gram-Schmidt applied twice per column
//                            (stable for a numerically full-rank Y), one CTA
//                            per shot, fp64; diag(R) > 0
// All work is small next to a gradient (nt * nrec * r multiply-adds, twice).
#include <algorithm>
#include <cstdio>

#include "tp_internal.h"
#include "tprobe.h"

namespace tp {

namespace {

constexpr int QR_RMAX = 32;
constexpr int QR_THREADS = 256;

__global__ void __launch_bounds__(128) qr_dtz_kernel(const float* __restrict__ D, const float* __restrict__ Z, int nt,
                                                     int nrec, int r, double* __restrict__ W) {
  const int s = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nrec) return;
  const float* Ds = D + (long long)s * nt * nrec;
  const float* Zs = Z + (long long)s * nt * r;
  double acc[QR_RMAX];
#pragma unroll
  for (int i = 0; i < QR_RMAX; ++i) acc[i] = 0.0;
  for (int t = 0; t < nt; ++t) {
    const double d = Ds[(long long)t * nrec + j];
#pragma unroll
    for (int i = 0; i < QR_RMAX; ++i)
      if (i < r) acc[i] += d * (double)__ldg(Zs + (long long)t * r + i);
  }
  double* Ws = W + ((long long)s * nrec + j) * r;
#pragma unroll
  for (int i = 0; i < QR_RMAX; ++i)
    if (i < r) Ws[i] = acc[i];
}

__global__ void __launch_bounds__(128) qr_dw_kernel(const float* __restrict__ D, const double* __restrict__ W, int nt,
                                                    int nrec, int r, double* __restrict__ Y) {
  const int s = blockIdx.y;
  const int t = blockIdx.x * 4 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (t >= nt) return;
  const float* Dt = D + ((long long)s * nt + t) * nrec;
  const double* Ws = W + (long long)s * nrec * r;
  double acc[QR_RMAX];
#pragma unroll
  for (int i = 0; i < QR_RMAX; ++i) acc[i] = 0.0;
  for (int j = lane; j < nrec; j += 32) {
    const double d = Dt[j];
#pragma unroll
    for (int i = 0; i < QR_RMAX; ++i)
      if (i < r) acc[i] += d * Ws[(long long)j * r + i];
  }
#pragma unroll
  for (int i = 0; i < QR_RMAX; ++i)
    for (int o = 16; o > 0; o >>= 1) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], o);
  if (lane < r) {
    double v = 0.0;
#pragma unroll
    for (int i = 0; i < QR_RMAX; ++i)
      if (i == lane) v = acc[i];
    Y[((long long)s * nt + t) * r + lane] = v;
  }
}

__device__ double qr_block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < QR_THREADS / 32; ++w) t += sh[w];  // same order in every thread
  __syncthreads();
  return t;
}

// Y is overwritten by the orthonormal Q (fp64); Qf receives it in fp32.
__global__ void __launch_bounds__(QR_THREADS) qr_cgs2_kernel(double* __restrict__ Y, int nt, int r,
                                                             float* __restrict__ Qf, int* err) {
  __shared__ double h[QR_RMAX];
  __shared__ double sh[QR_THREADS / 32];
  const int s = blockIdx.x;
  double* Ys = Y + (long long)s * nt * r;
  for (int k = 0; k < r; ++k) {
    double n0 = 0.0;
    for (int t = threadIdx.x; t < nt; t += QR_THREADS) n0 += Ys[(long long)t * r + k] * Ys[(long long)t * r + k];
    n0 = qr_block_sum(n0, sh);
    for (int pass = 0; pass < 2; ++pass) {  // twice is enough
      for (int i = 0; i < k; ++i) {
        double p = 0.0;
        for (int t = threadIdx.x; t < nt; t += QR_THREADS) p += Ys[(long long)t * r + i] * Ys[(long long)t * r + k];
        p = qr_block_sum(p, sh);
        if (threadIdx.x == 0) h[i] = p;
      }
      __syncthreads();
      for (int t = threadIdx.x; t < nt; t += QR_THREADS) {
        double v = Ys[(long long)t * r + k];
        for (int i = 0; i < k; ++i) v -= Ys[(long long)t * r + i] * h[i];
        Ys[(long long)t * r + k] = v;
      }
      __syncthreads();
    }
    double nn = 0.0;
    for (int t = threadIdx.x; t < nt; t += QR_THREADS) nn += Ys[(long long)t * r + k] * Ys[(long long)t * r + k];
    nn = qr_block_sum(nn, sh);
    // a column that vanished relative to its own size: numerically rank deficient
    const bool dep = !(nn > 1e-24 * n0) || nn <= 0.0;
    if (dep && threadIdx.x == 0) atomicOr(err, 4);
    const double inv = dep ? 0.0 : 1.0 / sqrt(nn);
    for (int t = threadIdx.x; t < nt; t += QR_THREADS) Ys[(long long)t * r + k] *= inv;
    __syncthreads();
  }
  for (long long e = threadIdx.x; e < (long long)nt * r; e += QR_THREADS) Qf[(long long)s * nt * r + e] = (float)Ys[e];
}

long long up256(long long b) { return (b + 255) / 256 * 256; }

struct QrLayout {
  size_t o_err, o_Z, o_W, o_Y, bytes;
};

QrLayout qr_layout(int nt, int nrec, int nshots, int r) {
  QrLayout L{};
  size_t cur = 0;
  L.o_err = cur; cur += 256;
  L.o_Z = cur; cur += up256((long long)nshots * nt * r * sizeof(float));
  L.o_W = cur; cur += up256((long long)nshots * nrec * r * sizeof(double));
  L.o_Y = cur; cur += up256((long long)nshots * nt * r * sizeof(double));
  L.bytes = cur;
  return L;
}

}  // namespace
}  // namespace tp

extern "C" {

size_t tp_qr_workspace_bytes(int nt, int nrec, int nshots, int r) {
  if (nt < 1 || nrec < 1 || nshots < 1 || r < 1 || r > tp::QR_RMAX) return 0;
  return tp::qr_layout(nt, nrec, nshots, r).bytes;
}

tp_status tp_qr_probes(const tp_probe* probe, int nt, int nrec, int nshots, const float* d_obs, float* Q, void* ws,
                       size_t ws_bytes, void* stream) {
  using namespace tp;
  char buf[160];
  auto bad = [&](tp_status st, const char* m) {
    snprintf(buf, sizeof(buf), "tp_qr_probes: %s", m);
    set_last_error(buf);
    return st;
  };
  if (!probe || !d_obs || !Q || !ws) return bad(TP_ERR_ARG, "NULL argument");
  if (probe->kind != TP_PROBE_RADEMACHER && probe->kind != TP_PROBE_GAUSSIAN)
    return bad(TP_ERR_ARG, "the random probes Z must be Rademacher or Gaussian");
  if (probe->r < 1 || probe->r > QR_RMAX) return bad(TP_ERR_ARG, "r must be in 1..32");
  if (nt < probe->r) return bad(TP_ERR_ARG, "nt must be >= r");
  if (nrec < 1 || nshots < 1) return bad(TP_ERR_ARG, "nrec and nshots must be >= 1");
  if (reinterpret_cast<uintptr_t>(ws) % 256) return bad(TP_ERR_ARG, "workspace must be 256-byte aligned");
  const QrLayout L = qr_layout(nt, nrec, nshots, probe->r);
  if (ws_bytes < L.bytes) return bad(TP_ERR_NOMEM, "workspace too small");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(ws);
  const int r = probe->r;
  cudaError_t e = cudaMemsetAsync(w + L.o_err, 0, 256, st);
  if (e == cudaSuccess) e = launch_probes(probe->kind, nt, r, probe->seed, 0, nshots, nullptr,
                                          reinterpret_cast<float*>(w + L.o_Z), st);
  if (e == cudaSuccess) {
    prof_before(5, st);
    qr_dtz_kernel<<<dim3((nrec + 127) / 128, nshots), 128, 0, st>>>(d_obs, reinterpret_cast<float*>(w + L.o_Z), nt,
                                                                     nrec, r, reinterpret_cast<double*>(w + L.o_W));
    qr_dw_kernel<<<dim3((nt + 3) / 4, nshots), 128, 0, st>>>(d_obs, reinterpret_cast<double*>(w + L.o_W), nt, nrec, r,
                                                             reinterpret_cast<double*>(w + L.o_Y));
    qr_cgs2_kernel<<<nshots, QR_THREADS, 0, st>>>(reinterpret_cast<double*>(w + L.o_Y), nt, r, Q,
                                                  reinterpret_cast<int*>(w + L.o_err));
    prof_after(5, st);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    snprintf(buf, sizeof(buf), "tp_qr_probes: %s", cudaGetErrorString(e));
    set_last_error(buf);
    return TP_ERR_CUDA;
  }
  return TP_OK;
}

}  // extern "C"
