// Internal declarations shared by the translation units of libtprobe.
// Not part of the public ABI (see include/tprobe.h).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

namespace tp {

// Halo width of every padded field in y and z: zero layers around the grid
// that make the Dirichlet boundary of the Laplacian free (radius R <= 4).
constexpr int H = 4;
// x halo: 32 zero columns, so that every row's interior starts on a 128-byte
// L2 line (row pitch a multiple of 32 floats).  Partial-line writes make the
// L2 fetch the rest of the line from DRAM; aligned rows avoid those fills.
// The right halo of a row is the left padding of the next row.
constexpr int HX = 32;
// x extents are padded to a multiple of this (tile widths of the sweeps).
constexpr int XALIGN = 128;
// y extents (3-D) are padded to a multiple of this.
constexpr int YALIGN = 16;

// Geometry of a padded field.  Grid node (z, y, x) lives at
//   (z + H) * plane + (y + yh) * px + (x + HX),  yh = H in 3-D, 0 in 2-D.
// Padding and halo cells are zero and never written by the kernels.
struct Layout {
  int ndim, nx, ny, nz;
  int px, py, pz;       // padded extents (py = 1 in 2-D)
  long long plane;      // py * px
  long long field;      // pz * plane + slack, rounded up to 64 floats (256 B)
  __host__ __device__ long long off(long long z, long long y, long long x) const {
    return (z + H) * plane + (y + (ndim == 3 ? H : 0)) * px + (x + HX);
  }
  __host__ __device__ long long off_flat(long long idx) const {  // dense (z*ny+y)*nx+x
    long long x = idx % nx, t = idx / nx;
    long long y = t % ny, z = t / ny;
    return off(z, y, x);
  }
};

Layout make_layout(int ndim, int nx, int ny, int nz);

// Centred second-derivative weights w[0..R] (Fornberg 1988) for order 2R.
// The sweeps use w[1..R] in the centred form sum_k w_k (sum of the 2 ndim
// neighbours at distance k - 2 ndim u), which equals ndim w[0] u + sum_k w_k
// (neighbours) because w[0] = -2 sum_k w_k, and leaves no zero-order term from
// the fp32 rounding of w[0].
struct Weights {
  float w[5];
  int R;
  int sw;       // absorbing layer width in cells (0: none)
  float samax;  // a = eta dt / 2 at the outermost node of the layer
};

// a = eta dt / 2 of the absorbing layer at node (z, y, x): samax ((sw - d)/sw)^2
// within sw cells of the bottom and side faces (the top z = 0 is the free
// surface), 0 elsewhere or without a layer.
__host__ __device__ inline float sponge_a(const Layout& L, const Weights& W, long long z, long long y, long long x) {
  if (W.sw <= 0) return 0.f;
  long long d = x < L.nx - 1 - x ? x : L.nx - 1 - x;
  const long long dz = L.nz - 1 - z;
  if (dz < d) d = dz;
  if (L.ndim == 3) {
    const long long dy = y < L.ny - 1 - y ? y : L.ny - 1 - y;
    if (dy < d) d = dy;
  }
  if (d >= W.sw) return 0.f;
  const float t = (float)(W.sw - d) / (float)W.sw;
  return W.samax * t * t;
}
Weights stencil_weights(int order);

// ---------------------------------------------------------------- stencil
enum StencilMode { MODE_STEP = 0, MODE_IMAGE = 1, MODE_INC = 2, MODE_STEP_IMG = 3 };

// A field of a "family": `nfields` consecutive padded fields starting at
// `base` (a ring of levels, a history, the accumulators...).  Shot s uses
// field f0 + s * fs (fs = 0: one field shared by all shots).
struct FieldRef {
  const float* base;
  int nfields;
  int f0;
  int fs;
  __host__ __device__ const float* ptr(const Layout& L, int shot) const {
    return base + (long long)(f0 + shot * fs) * L.field;
  }
};

// MODE_STEP : out = 2 src - p1 + p2 * S(src)          (leapfrog, p1 = older level, p2 = c2)
// MODE_INC  : w' = p1 + p2 * S(src), out = src + w', and w' is stored to out2
//             (the increment form: p1 = out2 = the increment u[t] - u[t-1])
// MODE_IMAGE: out = p2 + p1 * S(src)  (out may alias p2: accumulate)
// MODE_STEP_IMG (3-D only): MODE_STEP, and in the same sweep
//             gout = gin + src * S(img)  (the imaging condition of Eq. 3 on the
//             step's own source field; gout may alias gin)
// S(.) = the stencil sum without 1/h^2, in the centred form.  `out` is the shot-0 field,
// out_ss the per-shot stride in floats.
struct StencilArgs {
  FieldRef src, p1, p2;
  float* out;
  long long out_ss;
  int nshots;
  float* out2 = nullptr;     // MODE_INC: the increment field (same storage as p1)
  long long out2_ss = 0;
  FieldRef img{};            // MODE_STEP_IMG: the field under the imaging stencil
  FieldRef gin{};            // MODE_STEP_IMG: the accumulator read
  float* gout = nullptr;     // MODE_STEP_IMG: the accumulator written (shot 0), per-shot stride gout_ss
  long long gout_ss = 0;
};
cudaError_t launch_stencil(int mode, const Layout& L, const Weights& W, const StencilArgs& a,
                           cudaStream_t s, int* err);
// 4-D TMA map over a family of `nfields` consecutive padded fields of `esize`
// bytes per value (4: fp32, 2: bf16): dims (px, py, pz, nfields), box
// (box_x, box_y, 1, box_fields), no swizzle; encoded once per distinct key.
bool encode_field_map(const Layout& L, const void* base, long long nfields, int esize, int box_x, int box_y,
                      int box_fields, CUtensorMap* out);

// ---------------------------------------------------------------- 2-D cluster stepping
// Persistent 2-D time stepping (tp_sweep2d_cluster.cu): one thread-block
// cluster per shot holds the shot's levels in shared memory and runs nsteps
// steps per launch, with in-kernel injection (entries at one node summed in
// index order) and sampling.  Forward (dir = +1): step i forms level
// lev0 + i + 1 from lev0 + i and lev0 + i - 1; adjoint (dir = -1): level
// lev0 - i - 1 from lev0 - i and lev0 - i + 1.  Every new level is written to
// ring slot (level mod nslots) of its shot; the launch starts from the ring
// slots of lev0 and lev0 - dir (zero when fresh).  comp: double-float levels
// (low parts in bf16 slots eslots + shot * e_ss + (level mod 2) * field,
// written for the last two levels of a launch).  Injection: new level at
// inj_off[s][k] += inj_coef[s][k] * inj_val[s][new level + inj_shift][k];
// sampling: samp_out[s][new level + samp_shift][j] = new level at samp_off[s][j].
struct Cluster2dArgs {
  Layout L;
  Weights W;
  int nshots, comp, dir, lev0, nsteps, fresh;
  float* ring; int nslots; long long ring_ss;
  void* eslots; long long e_ss;
  const float* c2;
  const long long* inj_off; const float* inj_coef; int ninj;
  const float* inj_val; long long inj_val_ss; int inj_shift;
  const long long* samp_off; int nsamp; float* samp_out; long long samp_out_ss; int samp_shift;
};
cudaError_t launch_cluster2d(const Cluster2dArgs& a, cudaStream_t s);
// whether the cluster path can run a batch of this grid (2-D, no absorbing
// layer, a shot's bands fit one cluster, at most 1024 sources and receivers)
bool cluster2d_fits(const Layout& L, const Weights& W, int nshots, int nsrc, int nrec, bool comp);

// ---------------------------------------------------------------- probe GEMM
// P[s][i][x] += sum_{k < nlev} ring[s][(level0 + k) mod nslots][x] * Q[s][level0 + k + qshift][i]
// with Q rows outside [qlo, qhi] read as zero.  tcgen05 (kind::tf32) with a
// hi/lo split of the snapshots (and of Q when q_has_lo).
// The GEMM walks interior row segments of 128 points: M = nz * ny * nxt * 128
// with nxt = ceil(nx / 128); padding columns beyond nx inside a segment are
// zero in both operands and stay zero.
// Accumulator storage: acc = 0 fp32; 1 bf16; 2 bf16 value + bf16 compensation
// (the compensation of probe i is stored at element offset r * pstride after
// its value).  P, pstride and p_ss count elements of the storage type.
struct GemmArgs {
  Layout L;
  const float* ring; long long slot_stride; long long ring_ss; int nslots;
  int level0, nlev, qshift, qlo, qhi;
  const float* Q; int nt, r; long long q_ss;
  void* P; long long pstride; long long p_ss;  // P[s][i] at P + s*p_ss + i*pstride
  int acc;                 // 3: dot mode, G[s][x] += sum_i P[s][i][x] * tile[x, i] (P fp32, read only)
  float* G; long long g_ss;
  int nshots;
  int q_has_lo;
  int* err;
};
cudaError_t launch_probe_gemm(const GemmArgs& a, cudaStream_t s);
int gemm_kpad(int T);

// ---------------------------------------------------------------- misc kernels
cudaError_t launch_prep_c2(const Layout& L, const float* vel, double coef, float* c2, cudaStream_t s);
cudaError_t launch_vmax(const float* vel, long long n, unsigned int* out_bits, cudaStream_t s);
// dense node indices -> padded offsets, and injection coefficient dt^2 v^2 at each point
// (out-of-range indices get offset -1 and set bit 2 of *err)
cudaError_t launch_prep_points(const Layout& L, const Weights& W, const int64_t* idx, long long n, const float* vel,
                               double dt2, long long* off, float* cinj, int* err, cudaStream_t s);

// One thread per point of two independent sets, all shots:
//   sample: samp_out[s][t_s][j] = field_samp[s][samp_off[s][j]]           (j < nsamp)
//   inject: field_inj[s][inj_off[s][k]] += inj_coef[s][k] * inj_val[s][t_i][k]  (k < ninj)
//   srcacc (optional): acc[s][j] += sampled value * acc_val[s][t_a][j]
// Injection is deterministic: entries alone at their node (inj_alone[s][k])
// are added by their own thread, the others (inj_shared[s][0 .. inj_nshared[s]),
// in index order) by one thread per shot, one after the other.
struct PointArgs {
  int nshots;
  const float* field_samp; long long samp_ss;
  const long long* samp_off; int nsamp; float* samp_out; long long samp_out_ss;  // already offset to t
  float* field_inj; long long inj_ss;
  float* field_inj2; long long inj2_ss;  // optional second target (the increment field)
  const long long* inj_off; const float* inj_coef; int ninj;
  const float* inj_val; long long inj_val_ss;  // already offset to t
  const unsigned char* inj_alone; const int* inj_shared; const int* inj_nshared;
  double* acc; const float* acc_val; long long acc_val_ss;  // may be null
};
cudaError_t launch_point(const PointArgs& a, cudaStream_t s);
// alone / shared / nshared of a point set (per_shot entries per shot) from the
// padded offsets; cnt_scratch: nshots * field ints of scratch
cudaError_t launch_point_groups(const long long* off, int per_shot, int nshots, long long field, int* cnt_scratch,
                                unsigned char* alone, int* shared, int* nshared, cudaStream_t s);

cudaError_t launch_probes(int kind, int nt, int r, uint64_t seed, int shot0, int nshots,
                          const float* Z_user, float* Q, cudaStream_t s);

// res = d - dobs (in place over d), partial sums of res^2 into part[nblk]
cudaError_t launch_residual(float* d, const float* dobs, long long n, double* part, int nblk,
                            cudaStream_t s);
// part[block] = sum a^2 over a fixed grid-stride set
cudaError_t launch_sumsq(const float* a, long long n, double* part, int nblk, cudaStream_t s);
// out = scale * sum(part[0..nblk))  (fixed order; sqrt first if asked; NaN if *err & 1)
cudaError_t launch_finalize_sum(const double* part, int nblk, double scale, double* out,
                                int sqrt_result, const int* err, cudaStream_t s);
// grad[x] = -scale_h2 * vel[x]^2 * sum_s gacc[s][off(x)]   (times_v2 = 1)
// grad[x] = -scale_h2 * sum_s gacc[s][off(x)]              (times_v2 = 0)
cudaError_t launch_finish_grad(const Layout& L, const float* vel, const float* gacc, int nshots,
                               long long gacc_ss, float scale_h2, float* grad, cudaStream_t s, int times_v2 = 1);
// U[s][i][src_off[s][k]] += dt^2 v[src[s][k]]^2 * qbar[s][k][i]   (serial, fixed order)
cudaError_t launch_source_into_acc(const long long* src_off, const int64_t* src, const float* vel, double dt2,
                                   const float* qbar, int nsrc, int nshots, int r, float* U, long long u_ss,
                                   long long field, cudaStream_t s);
// fp32 copy of accumulator field i of every shot: out[s] = value (+ compensation)
cudaError_t launch_acc_to_f32(const void* P, int acc, int r, int i, long long field, int nshots, float* out,
                              long long out_ss, cudaStream_t s);
// grad <- grad * (-2 / vel^3): dJ/dv from dJ/dm (m = 1 / v^2)
cudaError_t launch_chain_velocity(const float* vel, float* grad, long long n, cudaStream_t s);
// image[x] = scale * sum_s sum_i <D P_s,i, D V_s,i>(x), D per tp_image_cond (tp_image.cu)
cudaError_t launch_image(const Layout& L, int order, float h, int cond, const float* P, long long p_ss,
                         const float* V, long long v_ss, int r, int nshots, float scale, float* image,
                         cudaStream_t s);
// qbar[s][k][i] = sum_{j=jlo}^{jhi} Q[s][j + qshift][i] * q[s][j][k]
cudaError_t launch_qbar(const float* Q, int nt, int r, const float* wav, int nsrc, int nshots,
                        int jlo, int jhi, int qshift, float* qbar, cudaStream_t s);
// grad[src[s][k]] += -scale * vel^2 * (probed: sum_i qbar[s][k][i] vbar[s][i][off]; full: srcacc[s][k])
// serial in a fixed order (deterministic when sources share a node)
cudaError_t launch_source_term(const Layout& L, const float* vel, const int64_t* src_dense,
                               const long long* src_off, int nsrc, int nshots, float scale,
                               const float* qbar, const void* V, int acc, int r, long long v_ss,
                               const double* srcacc, float* grad, cudaStream_t s);

// message returned by tp_last_error() on the calling thread
void set_last_error(const char* msg);

// Spin limit (SM clock cycles) of the bounded waits between the roles of the
// pipelined kernels, read at launch: the value set by tp_set_wait_limit, else
// DEFAULT_WAIT_CYCLES (about one second).  Waits that only drain a kernel's
// own copies before it exits always use the default.
constexpr long long DEFAULT_WAIT_CYCLES = 2000000000LL;
long long wait_limit_cycles();

// ---------------------------------------------------------------- profiling
void prof_before(int kind, cudaStream_t s);
void prof_after(int kind, cudaStream_t s);

// Raises kernel K's dynamic shared-memory limit to `bytes` (and, if asked,
// allows clusters above the portable size) on the current device, once per
// device: a function attribute belongs to the device's
// context, so a process that launches on several devices sets it on each.
// Thread-safe; devices beyond the first 64 are set on every call.
template <auto K>
cudaError_t smem_limit_once(int bytes, bool nonportable_cluster = false) {
  static std::atomic<unsigned long long> done{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = dev < 64 ? 1ULL << dev : 0ULL;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess && nonportable_cluster)
    e = cudaFuncSetAttribute(K, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

}  // namespace tp
