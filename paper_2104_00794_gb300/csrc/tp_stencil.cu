// Leapfrog stencil sweeps (Algorithm 1 lines 1 and 5, operators f and f^T)
// and the stencil-form imaging sweep for 2-D padded fields, and the dispatch
// of every sweep (3-D ones run in tp_sweep3d_tma.cu).
//
// Design (~16 B per grid point per step; a 2-D batch usually sits in L2):
//   * every warp owns an x strip of 128 points and sweeps a chunk of z rows;
//     each lane owns 4 consecutive x points (float4 access);
//   * the z neighbours of the lane's points live in a register queue of
//     2R+1 float4 values, the current row (with its x halo) in shared
//     memory, so each haloed value is read from L2/HBM about once per sweep;
//   * all global loads of row z+1 (queue head, halo, older level,
//     coefficient) are issued before row z is computed;
//   * zero halo layers of the padded layout supply the Dirichlet boundary,
//     so no load is predicated.
#include <algorithm>

#include "tp_internal.h"

namespace tp {

namespace {

// pointer + per-shot stride form used by the plain sweeps
struct PlainArgs {
  const float* src;  long long src_ss;
  const float* p1;   long long p1_ss;
  const float* p2;   long long p2_ss;
  float* out;        long long out_ss;
  int nshots;
  float* out2;       long long out2_ss;  // MODE_INC: increment field
};

__device__ __forceinline__ float4 ld4(const float* base, long long idx) {
  return __ldg(reinterpret_cast<const float4*>(base + idx));
}

// returns the new value; in MODE_INC also the new increment through *inc.
// a: damping of the absorbing layer at this node (0 outside it, where the
// undamped expressions run unchanged).
template <int MODE>
__device__ __forceinline__ float epilogue(float c, float s, float p1, float p2, float* inc, float a) {
  if (MODE == MODE_STEP) {
    if (a == 0.f) return fmaf(p2, s, 2.0f * c - p1);
    return fmaf(p2, s, 2.0f * c - (1.0f - a) * p1) / (1.0f + a);
  }
  if (MODE == MODE_INC) {
    *inc = a == 0.f ? fmaf(p2, s, p1) : fmaf(p2, s, (1.0f - a) * p1) / (1.0f + a);
    return c + *inc;
  }
  return fmaf(p1, s, p2);
}

__device__ __forceinline__ float comp(const float4& v, int p) {
  return p == 0 ? v.x : (p == 1 ? v.y : (p == 2 ? v.z : v.w));
}

__device__ __forceinline__ void store_masked(float* out, long long idx, float4 v, int x, int nx) {
  if (x + 3 < nx) {
    *reinterpret_cast<float4*>(out + idx) = v;
  } else {
    if (x + 0 < nx) out[idx + 0] = v.x;
    if (x + 1 < nx) out[idx + 1] = v.y;
    if (x + 2 < nx) out[idx + 2] = v.z;
    if (x + 3 < nx) out[idx + 3] = v.w;
  }
}

// ------------------------------------------------------------------ 2-D
constexpr int W2 = 4;  // warps per CTA, each an independent (x strip, z chunk)

template <int R, int MODE, bool DAMP>
__global__ void __launch_bounds__(32 * W2)
sweep2d(Layout L, Weights W, PlainArgs a, int bz, int nzc, int nxt, int nwarps) {
  __shared__ float4 sm[W2][32 + 2];
  const int lane = threadIdx.x, wi = threadIdx.y;
  const int gw = blockIdx.x * W2 + wi;
  if (gw >= nwarps) return;
  const int xt = gw % nxt;
  const int zc = (gw / nxt) % nzc;
  const int shot = gw / (nxt * nzc);
  const int x0 = xt * 128, x = x0 + 4 * lane;
  const int zb = zc * bz, ze = min(L.nz, zb + bz);
  if (zb >= ze) return;

  const float* src = a.src + shot * a.src_ss;
  const float* p1 = a.p1 + shot * a.p1_ss;
  const float* p2 = a.p2 + shot * a.p2_ss;
  float* out = a.out + shot * a.out_ss;
  const long long pl = L.px;  // row pitch (plane == px in 2-D)
  const long long colc = (long long)(x + HX) + (long long)H * pl;
  const long long colxl = (long long)(x0 - 4 + HX) + (long long)H * pl;
  const long long colxr = (long long)(x0 + 128 + HX) + (long long)H * pl;
  const bool hxl = lane == 0, hxr = lane == 31;

  float4 q[2 * R + 1];
#pragma unroll
  for (int k = 0; k < 2 * R; ++k) q[k] = ld4(src, colc + (long long)(zb - R + k) * pl);
  float4 nq = ld4(src, colc + (long long)(zb + R) * pl);
  float4 n1 = ld4(p1, colc + (long long)zb * pl);
  float4 n2 = ld4(p2, colc + (long long)zb * pl);
  float4 nhx = make_float4(0.f, 0.f, 0.f, 0.f);
  if (hxl) nhx = ld4(src, colxl + (long long)zb * pl);
  if (hxr) nhx = ld4(src, colxr + (long long)zb * pl);

  for (int z = zb; z < ze; ++z) {
    q[2 * R] = nq;
    sm[wi][lane + 1] = q[R];
    if (hxl) sm[wi][0] = nhx;
    if (hxr) sm[wi][33] = nhx;
    const float4 c1 = n1, c2 = n2;
    if (z + 1 < ze) {
      const long long zo = (long long)(z + 1) * pl;
      nq = ld4(src, colc + zo + (long long)R * pl);
      n1 = ld4(p1, colc + zo);
      n2 = ld4(p2, colc + zo);
      if (hxl) nhx = ld4(src, colxl + zo);
      if (hxr) nhx = ld4(src, colxr + zo);
    }
    __syncwarp();
    const float4 xl = sm[wi][lane], xc = sm[wi][lane + 1], xr = sm[wi][lane + 2];
    const float v[12] = {xl.x, xl.y, xl.z, xl.w, xc.x, xc.y, xc.z, xc.w, xr.x, xr.y, xr.z, xr.w};
    // centred form (see tp_sweep3d_tma.cu): sum_k w_k (neighbour sum - 4u), the -4u
    // folded into one FMA; two points per packed fp32x2 instruction, each lane the
    // scalar operation in the same order
    float2 s2[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    const float2 m4 = make_float2(-4.f, -4.f);
#pragma unroll
    for (int k = 1; k <= R; ++k) {
      const float4 zp = q[R + k], zm = q[R - k];
      const float2 wk = make_float2(W.w[k], W.w[k]);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int p = 2 * h;
        const float2 c = make_float2(v[4 + p], v[5 + p]);
        const float2 xs = __fadd2_rn(make_float2(v[4 + p + k], v[5 + p + k]), make_float2(v[4 + p - k], v[5 + p - k]));
        const float2 zs = __fadd2_rn(h ? make_float2(zp.z, zp.w) : make_float2(zp.x, zp.y),
                                     h ? make_float2(zm.z, zm.w) : make_float2(zm.x, zm.y));
        s2[h] = __ffma2_rn(wk, __ffma2_rn(m4, c, __fadd2_rn(xs, zs)), s2[h]);
      }
    }
    const float s4[4] = {s2[0].x, s2[0].y, s2[1].x, s2[1].y};
    float res[4], inc[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const float ad = (DAMP && MODE != MODE_IMAGE) ? sponge_a(L, W, z, 0, x + p) : 0.f;
      res[p] = epilogue<MODE>(v[4 + p], s4[p], comp(c1, p), comp(c2, p), &inc[p], ad);
    }
    if (x < L.nx) {
      store_masked(out, colc + (long long)z * pl, make_float4(res[0], res[1], res[2], res[3]), x, L.nx);
      if (MODE == MODE_INC)
        store_masked(a.out2 + shot * a.out2_ss, colc + (long long)z * pl, make_float4(inc[0], inc[1], inc[2], inc[3]), x, L.nx);
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < 2 * R; ++k) q[k] = q[k + 1];
  }
}

// SM count of the current device, cached per device (thread-safe)
int num_sms() {
  static std::atomic<int> cache[64];
  int dev = 0;
  cudaGetDevice(&dev);
  int n = dev >= 0 && dev < 64 ? cache[dev].load(std::memory_order_relaxed) : 0;
  if (n <= 0) {
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
    if (dev >= 0 && dev < 64) cache[dev].store(n, std::memory_order_relaxed);
  }
  return n;
}

template <int R, int MODE>
cudaError_t launch2d(const Layout& L, const Weights& W, const PlainArgs& a, cudaStream_t s) {
  const int nxt = (L.nx + 127) / 128;
  const long long strips = (long long)nxt * a.nshots;
  const long long target = 16LL * W2 * num_sms();  // warps
  int nzc = (int)std::max<long long>(1, (target + strips - 1) / strips);
  nzc = std::min(nzc, std::max(1, L.nz / 8));
  const int bz = (L.nz + nzc - 1) / nzc;
  nzc = (L.nz + bz - 1) / bz;
  const int nwarps = nxt * nzc * a.nshots;
  dim3 grid((nwarps + W2 - 1) / W2), block(32, W2);
  if (MODE != MODE_IMAGE && W.sw > 0) sweep2d<R, MODE, true><<<grid, block, 0, s>>>(L, W, a, bz, nzc, nxt, nwarps);
  else sweep2d<R, MODE, false><<<grid, block, 0, s>>>(L, W, a, bz, nzc, nxt, nwarps);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sweep3d_tma(int mode, const Layout& L, const Weights& W, const StencilArgs& a, cudaStream_t s,
                               int* err);

// 3-D sweeps use the TMA-pipelined kernel (tp_sweep3d_tma.cu), 2-D ones the
// warp-strip kernel above.
cudaError_t launch_stencil(int mode, const Layout& L, const Weights& W, const StencilArgs& sa,
                           cudaStream_t s, int* err) {
  // TP_KERNEL_IMAGING / TP_KERNEL_STEP_IMAGING / TP_KERNEL_STENCIL
  const int kind = mode == MODE_IMAGE ? 1 : (mode == MODE_STEP_IMG ? 6 : 0);
  if (mode == MODE_STEP_IMG && L.ndim != 3) return cudaErrorInvalidValue;  // 3-D sweep only
  prof_before(kind, s);
  cudaError_t e;
  if (L.ndim == 3) {
    e = launch_sweep3d_tma(mode, L, W, sa, s, err);
  } else {
    PlainArgs a{sa.src.ptr(L, 0), (long long)sa.src.fs * L.field, sa.p1.ptr(L, 0), (long long)sa.p1.fs * L.field,
                sa.p2.ptr(L, 0), (long long)sa.p2.fs * L.field, sa.out, sa.out_ss, sa.nshots, sa.out2, sa.out2_ss};
#define TP_DISPATCH(FN, RR)                                                   \
  (mode == MODE_STEP ? FN<RR, MODE_STEP>(L, W, a, s)                          \
                     : (mode == MODE_INC ? FN<RR, MODE_INC>(L, W, a, s) : FN<RR, MODE_IMAGE>(L, W, a, s)))
    e = W.R == 4 ? TP_DISPATCH(launch2d, 4) : TP_DISPATCH(launch2d, 2);
#undef TP_DISPATCH
  }
  prof_after(kind, s);
  return e;
}

}  // namespace tp
