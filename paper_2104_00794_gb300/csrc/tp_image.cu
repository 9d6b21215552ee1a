// Imaging conditions applied to the probed wavefields (§Imaging conditions,
// Eq. 5: Q^T (D_x u) = D_x (Q^T u) for an operator D_x that acts on space
// only).  Instead of applying D_x to all nt snapshots of u and lambda, it is
// applied to the r probed fields P_i = sum_j Q[j+1, i] u[j] and
// V_i = sum_k Q[k, i] lambda[k]:
//
//   image(x) = scale * sum_shots sum_i < D P_i(x), D V_i(x) >
//
//   TP_IMAGE_CORRELATION  D = identity: the cross-correlation image
//                         sum_j u[j] lambda[j+1], probed;
//   TP_IMAGE_GRADIENT     D = the spatial gradient (centred first
//                         differences of the grid's order, 1/h), the
//                         product summed over the axes: the spatial term
//                         grad u . grad lambda of the inverse-scattering
//                         imaging condition, probed.
//
// One thread per grid point; the fields' zero halos are the values outside
// the grid.  The work is r x shots field pairs, once per image, next to
// nt x shots applications of D without probing.
#include "tp_internal.h"
#include "tprobe.h"

namespace tp {

namespace {

struct ImageArgs {
  Layout L;
  int R;
  float cd[4];  // centred first-derivative weights c_1..c_R divided by h
  int cond;
  const float* P;
  long long p_ss;  // per shot, floats
  const float* V;
  long long v_ss;
  int r, nshots;
  float scale;
  float* image;  // dense [nz][ny][nx]
};

__device__ __forceinline__ float dfirst(const float* f, long long o, long long stride, const float* cd, int R) {
  float d = 0.f;
#pragma unroll 4
  for (int k = 1; k <= R; ++k) d = fmaf(cd[k - 1], f[o + k * stride] - f[o - k * stride], d);
  return d;
}

__global__ void image_kernel(ImageArgs a) {
  const long long n = (long long)a.L.nx * a.L.ny * a.L.nz;
  const long long sx = 1, sy = a.L.px, sz = a.L.plane;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long o = a.L.off_flat(idx);
    float acc = 0.f;
    for (int s = 0; s < a.nshots; ++s) {
      const float* Ps = a.P + s * a.p_ss;
      const float* Vs = a.V + s * a.v_ss;
      for (int i = 0; i < a.r; ++i) {
        const float* p = Ps + (long long)i * a.L.field;
        const float* v = Vs + (long long)i * a.L.field;
        if (a.cond == TP_IMAGE_CORRELATION) {
          acc = fmaf(p[o], v[o], acc);
        } else {
          acc = fmaf(dfirst(p, o, sz, a.cd, a.R), dfirst(v, o, sz, a.cd, a.R), acc);
          if (a.L.ndim == 3) acc = fmaf(dfirst(p, o, sy, a.cd, a.R), dfirst(v, o, sy, a.cd, a.R), acc);
          acc = fmaf(dfirst(p, o, sx, a.cd, a.R), dfirst(v, o, sx, a.cd, a.R), acc);
        }
      }
    }
    a.image[idx] = a.scale * acc;
  }
}

}  // namespace

cudaError_t launch_image(const Layout& L, int order, float h, int cond, const float* P, long long p_ss,
                         const float* V, long long v_ss, int r, int nshots, float scale, float* image,
                         cudaStream_t s) {
  ImageArgs a{};
  a.L = L;
  a.R = order / 2;
  // centred first-derivative weights (Fornberg 1988, Table 1)
  const double w4[2] = {2.0 / 3.0, -1.0 / 12.0};
  const double w8[4] = {4.0 / 5.0, -1.0 / 5.0, 4.0 / 105.0, -1.0 / 280.0};
  for (int k = 0; k < a.R; ++k) a.cd[k] = (float)((order == 4 ? w4[k] : w8[k]) / (double)h);
  a.cond = cond;
  a.P = P;
  a.p_ss = p_ss;
  a.V = V;
  a.v_ss = v_ss;
  a.r = r;
  a.nshots = nshots;
  a.scale = scale;
  a.image = image;
  const long long n = (long long)L.nx * L.ny * L.nz;
  const int threads = 256;
  const long long blocks = std::max<long long>(1, std::min<long long>((n + threads - 1) / threads, 8192));
  prof_before(5, s);
  image_kernel<<<(unsigned)blocks, threads, 0, s>>>(a);
  prof_after(5, s);
  return cudaGetLastError();
}

}  // namespace tp
