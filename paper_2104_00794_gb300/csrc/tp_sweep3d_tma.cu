// 3-D leapfrog / imaging sweep with TMA-staged planes (sm_103a).
//
// Algorithm 1 lines 1 and 5 (operators f and f^T) are one 2k-order star
// stencil per time step: out = 2u - u_old + c2 * S(u), S(u) = sum_k w_k times
// the sum over the six neighbours at distance k of (neighbour - u).  The
// kernel is HBM-bound (16 B per point: read u, u_old, c2; write out).  Design:
//   * work items = (64 x 16 x-y tile, shot, z chunk); each tile column is cut
//     into as many equal z chunks as keep one wave of 2 CTAs per SM busy, and
//     items are ordered chunk-major, so neighbouring tiles are swept at the
//     same depths at the same time and their shared halo planes hit in L2
//     (a balanced linear split over (tile, z) left neighbours at different
//     depths: the halo re-reads went to DRAM, 1.44x the algorithmic reads);
//   * one producer thread streams, with cp.async.bulk.tensor (4-D tensor
//     maps over the padded field families), the haloed u plane
//     [16+2R][64+8] and the u_old / c2 planes [16][64] into a ring of shared
//     memory stages guarded by mbarriers (full: TMA transaction bytes,
//     empty: one arrival per consumer warp), R+1+3 u planes deep so three
//     planes are in flight while R+1 are resident;
//   * 256 consumer threads own 4 consecutive x points each; the z neighbours
//     live in a register queue of 2R+1 float4, x/y neighbours are read from
//     the resident centre plane (x halo from the box, zero halo layers from
//     the padded layout), so every value crosses HBM about once per step;
//   * the full-storage adjoint (MODE_STEP_IMG) also stages the history level
//     u[j] (haloed, on the u stages' barriers) and the gradient accumulator (on
//     the u_old / c2 stages'), keeps u[j]'s z neighbours in a second register
//     queue, and adds the imaging term of Eq. 3, lambda[j+1] * S(u[j]), in the
//     same pass: 28 B per point instead of 16 + 16 in two sweeps, one CTA per SM;
//   * every wait is bounded (clock64); on a timeout the CTA sets bit 0 of
//     *err, stops issuing, drains its own copies (bounded) and exits.
#include <cuda.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "tp_internal.h"

namespace tp {

namespace {

// lookahead of the fused step-and-imaging sweep, which runs one CTA per SM
// (164 registers a thread at order 8; at two CTAs per SM the 96-register cap
// spilled 1.7 KB a thread): full-storage gradient of 256^3, nt = 2000 on
// GB300: 2 planes 326.9 ms, 3 planes 314.0 ms, 5 planes 311.7 ms
constexpr int IMG_LA = 5;

// Tile BX x BY (BX/4 * BY == NCONS) and LA planes of lookahead.  IMG: the
// fused step-and-imaging sweep, with a second haloed field (its planes share
// the u stages' barriers) and the accumulator (sharing the u_old / c2 stages').
template <int R, int BX_, int BY_, int LA_, bool IMG_ = false>
struct Cfg {
  static constexpr int BX = BX_, BY = BY_, LA = LA_;
  static constexpr bool IMG = IMG_;
  static constexpr int NCONS = (BX / 4) * BY;  // consumer threads, 4 x points each
  static constexpr int NTHREADS = NCONS + 32;  // + one producer warp
  static_assert(NCONS % 32 == 0 && NCONS <= 992, "whole consumer warps");
  static constexpr int NSU = R + 1 + LA;  // u stages
  static constexpr int NSP = LA + 1;      // u_old / c2 stages
  static constexpr int NFU = IMG ? 2 : 1, NFP = IMG ? 3 : 2;  // fields per u stage, per u_old / c2 stage
  static constexpr int UW = BX + 8, UH = BY + 2 * R;
  static constexpr int UFL = UW * UH, PFL = BX * BY;
  static constexpr uint32_t UBYTES = UFL * 4, PBYTES = PFL * 4;
  static constexpr size_t BAR_OFF = (size_t)(NFU * NSU * UFL + NFP * NSP * PFL) * 4;
  static constexpr size_t SMEM = BAR_OFF + (size_t)(2 * NSU + 2 * NSP) * 8 + 16;
};

struct TmaArgs {
  Layout L;
  Weights W;
  int f_src, fs_src, f_p1, fs_p1, f_p2, fs_p2;
  int f_img, fs_img, f_g, fs_g;  // IMG: the imaged field and the accumulator read
  float* gout;                   // IMG: the accumulator written
  long long gout_ss;
  float* out;
  long long out_ss;
  float* out2;
  long long out2_ss;
  int nshots, ntx, nty;
  int nzc, zchunk;  // each tile column is cut into nzc chunks of zchunk planes
  long long items;  // tiles x shots x nzc work items
  long long spin;   // limit of the role waits (cycles); the drain waits use DEFAULT_WAIT_CYCLES
  int* err;
};

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint32_t b, uint32_t n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(b), "r"(n));
}
__device__ __forceinline__ void bar_expect_tx(uint32_t b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bar_arrive(uint32_t b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(b) : "memory");
}
__device__ __forceinline__ bool bar_try(uint32_t b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(b), "r"(parity)
      : "memory");
  return ok != 0;
}
// non-blocking probe of a phase (mbarrier.try_wait may suspend the thread in
// hardware until the phase completes, longer than a short wait limit)
__device__ __forceinline__ bool bar_test(uint32_t b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(b), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait; false on timeout or when another role has aborted.  With the
// default limit it polls with try_wait (the thread sleeps in hardware between
// polls); with a shorter one, set through tp_set_wait_limit, with test_wait,
// so that the limit is what ends the wait.
__device__ __forceinline__ bool bar_wait(uint32_t b, uint32_t parity, volatile int* abort_flag, long long limit) {
  const bool quick = limit < DEFAULT_WAIT_CYCLES;
  if (quick ? bar_test(b, parity) : bar_try(b, parity)) return true;
  const long long t0 = clock64();
  while (!(quick ? bar_test(b, parity) : bar_try(b, parity))) {
    if (*abort_flag) return false;
    if (clock64() - t0 > limit) {
      *abort_flag = 1;
      return false;
    }
  }
  return true;
}
// the same for a consumer warp: one decision for the whole warp, so that no
// lane leaves the plane loop while the others reach a warp-wide sync
__device__ __forceinline__ bool warp_wait(uint32_t b, uint32_t parity, volatile int* abort_flag, long long limit) {
  return __all_sync(0xffffffffu, bar_wait(b, parity, abort_flag, limit));
}
__device__ __forceinline__ void tma4(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                     uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}

__device__ __forceinline__ float comp(const float4& v, int p) {
  return p == 0 ? v.x : (p == 1 ? v.y : (p == 2 ? v.z : v.w));
}

struct Seg {
  int shot, x0, y0, z0, z1;
};

// Work item -> (tile, shot, z chunk).  Items are ordered chunk-major, so a
// wave of CTAs sweeps the same depths of neighbouring tiles at the same time
// and the x/y halo planes one CTA reads are still in L2 for its neighbours.
template <int BX, int BY>
__device__ __forceinline__ Seg segment(const TmaArgs& a, long long item) {
  const long long per = (long long)a.ntx * a.nty * a.nshots;
  const int zc = (int)(item / per);
  const long long rest = item % per;
  Seg s;
  s.shot = (int)(rest / ((long long)a.ntx * a.nty));
  const int t = (int)(rest % ((long long)a.ntx * a.nty));
  s.x0 = (t % a.ntx) * BX;
  s.y0 = (t / a.ntx) * BY;
  s.z0 = zc * a.zchunk;
  s.z1 = min(a.L.nz, s.z0 + a.zchunk);
  return s;
}

// S of Eq. 1 at the 4 consecutive x points of one consumer thread: v gets the
// centre row's 12 values around them (x - 4 .. x + 7), s4 the four sums.
// Uc: the resident centre plane (x/y neighbours), q: the z queue (q[R] is the
// centre plane's own float4).
// Centred form: S(u) = sum_k w_k (sum of the 6 neighbours at distance k - 6u), the
// -6u folded into one FMA per k (one rounding: fma(-6, u, sum), exact product).  It
// equals w_0 * 3u + sum_k w_k (neighbours) for exact weights, but carries no w_0
// term: with fp32-rounded weights the plain sum form keeps a spurious zero-order
// term that makes long runs drift, while here a constant field leaves only the
// rounding of its 6-fold sum, of either sign.  7 operations per k instead of the
// 12 of the per-neighbour difference form (u[+k] - u) + (u[-k] - u), at the same
// accuracy after thousands of steps.
// Two points per instruction with the packed fp32x2 FMA / ADD: each lane is the
// IEEE round-to-nearest operation of the scalar form, in the same order.
template <int R, int RW>
__device__ __forceinline__ void star4(const float4* Uc, const float4 (&q)[2 * R + 1], int cidx, const Weights& W,
                                      float (&v)[12], float (&s4)[4]) {
  const float4 xl = Uc[cidx - 1], xc = Uc[cidx], xr = Uc[cidx + 1];
  v[0] = xl.x; v[1] = xl.y; v[2] = xl.z; v[3] = xl.w;
  v[4] = xc.x; v[5] = xc.y; v[6] = xc.z; v[7] = xc.w;
  v[8] = xr.x; v[9] = xr.y; v[10] = xr.z; v[11] = xr.w;
  float2 s2[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  const float2 m6 = make_float2(-6.f, -6.f);
#pragma unroll
  for (int k = 1; k <= R; ++k) {
    const float4 yp = Uc[cidx + k * RW], ym = Uc[cidx - k * RW];
    const float4 zp = q[R + k], zm = q[R - k];
    const float2 wk = make_float2(W.w[k], W.w[k]);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int p = 2 * h;
      const float2 c = make_float2(v[4 + p], v[5 + p]);
      const float2 xs = __fadd2_rn(make_float2(v[4 + p + k], v[5 + p + k]), make_float2(v[4 + p - k], v[5 + p - k]));
      const float2 ys = __fadd2_rn(h ? make_float2(yp.z, yp.w) : make_float2(yp.x, yp.y),
                                   h ? make_float2(ym.z, ym.w) : make_float2(ym.x, ym.y));
      const float2 zs = __fadd2_rn(h ? make_float2(zp.z, zp.w) : make_float2(zp.x, zp.y),
                                   h ? make_float2(zm.z, zm.w) : make_float2(zm.x, zm.y));
      const float2 t = __ffma2_rn(m6, c, __fadd2_rn(__fadd2_rn(xs, ys), zs));
      s2[h] = __ffma2_rn(wk, t, s2[h]);
    }
  }
  s4[0] = s2[0].x; s4[1] = s2[0].y; s4[2] = s2[1].x; s4[3] = s2[1].y;
}

// DAMP: the grid has an absorbing layer (the undamped instantiation carries
// no trace of it)
template <int R, int MODE, class C, bool DAMP>
__global__ void __launch_bounds__(C::NTHREADS, C::SMEM + 1024 <= 114 * 1024 ? 2 : 1)
sweep3d_tma(const __grid_constant__ CUtensorMap mU, const __grid_constant__ CUtensorMap mP1,
            const __grid_constant__ CUtensorMap mP2, const __grid_constant__ CUtensorMap mI,
            const __grid_constant__ CUtensorMap mG, TmaArgs a) {
  constexpr int BX = C::BX, BY = C::BY;
  extern __shared__ __align__(128) unsigned char smem[];
  float* sU = reinterpret_cast<float*>(smem);
  float* sI = sU + C::NSU * C::UFL;  // IMG only
  float* sP1 = sU + C::NFU * C::NSU * C::UFL;
  float* sP2 = sP1 + C::NSP * C::PFL;
  float* sG = sP2 + C::NSP * C::PFL;  // IMG only
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::BAR_OFF);
  const uint32_t fullU = su32(bars), emptyU = fullU + 8 * C::NSU;
  const uint32_t fullP = emptyU + 8 * C::NSU, emptyP = fullP + 8 * C::NSP;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + 2 * C::NSU + 2 * C::NSP);

  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int s = 0; s < C::NSU; ++s) {
      bar_init(fullU + 8 * s, 1);
      bar_init(emptyU + 8 * s, C::NCONS / 32);
    }
    for (int s = 0; s < C::NSP; ++s) {
      bar_init(fullP + 8 * s, 1);
      bar_init(emptyP + 8 * s, C::NCONS / 32);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();


  if (tid >= C::NCONS) {
    // ------------------------------------------------------------ producer
    if (tid != C::NCONS) return;
    uint32_t ku = 0, kp = 0;
    bool ok = true;
    for (long long item = blockIdx.x; item < a.items && ok; item += gridDim.x) {
      const Seg sg = segment<BX, BY>(a, item);
      const int nzs = sg.z1 - sg.z0;
      if (nzs <= 0) continue;
      const int fu = a.f_src + sg.shot * a.fs_src, f1 = a.f_p1 + sg.shot * a.fs_p1, f2 = a.f_p2 + sg.shot * a.fs_p2;
      const int fi = a.f_img + sg.shot * a.fs_img, fg = a.f_g + sg.shot * a.fs_g;
      for (int k = 0; k < nzs + 2 * R && ok; ++k) {
        const int su = ku % C::NSU;
        if (ku >= (uint32_t)C::NSU && !bar_wait(emptyU + 8 * su, ((ku / C::NSU) - 1) & 1, abort_flag, a.spin)) {
          ok = false;
          break;
        }
        bar_expect_tx(fullU + 8 * su, C::NFU * C::UBYTES);
        // haloed u plane z = z0 - R + k: padded x from x0 - 4 + HX, y from y0 - R + H
        tma4(su32(sU + su * C::UFL), &mU, sg.x0 - 4 + HX, sg.y0 - R + H, sg.z0 - R + k + H, fu, fullU + 8 * su);
        if (C::IMG)  // the imaged field's plane, same box
          tma4(su32(sI + su * C::UFL), &mI, sg.x0 - 4 + HX, sg.y0 - R + H, sg.z0 - R + k + H, fi, fullU + 8 * su);
        ++ku;
        if (k >= 2 * R) {
          const int j = k - 2 * R;
          const int sp = kp % C::NSP;
          if (kp >= (uint32_t)C::NSP && !bar_wait(emptyP + 8 * sp, ((kp / C::NSP) - 1) & 1, abort_flag, a.spin)) {
            ok = false;
            break;
          }
          bar_expect_tx(fullP + 8 * sp, C::NFP * C::PBYTES);
          tma4(su32(sP1 + sp * C::PFL), &mP1, sg.x0 + HX, sg.y0 + H, sg.z0 + j + H, f1, fullP + 8 * sp);
          tma4(su32(sP2 + sp * C::PFL), &mP2, sg.x0 + HX, sg.y0 + H, sg.z0 + j + H, f2, fullP + 8 * sp);
          if (C::IMG) tma4(su32(sG + sp * C::PFL), &mG, sg.x0 + HX, sg.y0 + H, sg.z0 + j + H, fg, fullP + 8 * sp);
          ++kp;
        }
      }
    }
    if (!ok) atomicOr(a.err, 1);
    // drain: wait (bounded) until every copy this thread issued has landed
    for (int s = 0; s < C::NSU; ++s) {
      const uint32_t uses = ku > (uint32_t)s ? (ku - 1 - s) / C::NSU + 1 : 0;
      if (uses) {
        const long long t0 = clock64();
        while (!bar_try(fullU + 8 * s, (uses - 1) & 1) && clock64() - t0 < DEFAULT_WAIT_CYCLES) {}
      }
    }
    for (int s = 0; s < C::NSP; ++s) {
      const uint32_t uses = kp > (uint32_t)s ? (kp - 1 - s) / C::NSP + 1 : 0;
      if (uses) {
        const long long t0 = clock64();
        while (!bar_try(fullP + 8 * s, (uses - 1) & 1) && clock64() - t0 < DEFAULT_WAIT_CYCLES) {}
      }
    }
    return;
  }

  // -------------------------------------------------------------- consumers
  const int tx = tid % (BX / 4), ty = tid / (BX / 4), lane = tid & 31;
  constexpr int RW = C::UW / 4;  // float4 per staged row
  const float4* U4 = reinterpret_cast<const float4*>(sU);
  const float4* I4 = reinterpret_cast<const float4*>(sI);
  uint32_t ku = 0, kp = 0;
  bool ok = true;
  for (long long item = blockIdx.x; item < a.items && ok; item += gridDim.x) {
    const Seg sg = segment<BX, BY>(a, item);
    const int nzs = sg.z1 - sg.z0;
    if (nzs <= 0) continue;
    const int x = sg.x0 + 4 * tx, y = sg.y0 + ty;
    float* out = a.out + sg.shot * a.out_ss;
    float* out2 = MODE == MODE_INC ? a.out2 + sg.shot * a.out2_ss : nullptr;
    float* gout = C::IMG ? a.gout + sg.shot * a.gout_ss : nullptr;
    const int cidx = (ty + R) * RW + tx + 1;  // own float4 in a staged u plane
    float4 q[2 * R + 1], qi[2 * R + 1];  // qi: the imaged field's z neighbours (IMG)
    // prologue: planes z0-R .. z0+R-1 fill the queue; the first R are released
#pragma unroll
    for (int k = 0; k < 2 * R; ++k) {
      const uint32_t kk = ku + k, s = kk % C::NSU;
      if (!warp_wait(fullU + 8 * s, (kk / C::NSU) & 1, abort_flag, a.spin)) { ok = false; break; }
      q[k] = U4[s * (C::UFL / 4) + cidx];
      if (C::IMG) qi[k] = I4[s * (C::UFL / 4) + cidx];
      if (k < R) {
        __syncwarp();
        if (lane == 0) bar_arrive(emptyU + 8 * s);
      }
    }
    // unrolled by the queue length (leapfrog and imaging sweeps): the register queue is
    // renamed instead of shifted (32 moves per plane; 63.6 -> 59.5 us per 256^3 step)
#pragma unroll((MODE != MODE_INC && !DAMP) ? 2 * R + 1 : 1)
    for (int j = 0; j < nzs && ok; ++j) {
      const uint32_t kc = ku + j + R, kn = ku + j + 2 * R, kq = kp + j;
      const uint32_t sc = kc % C::NSU, sn = kn % C::NSU, sp = kq % C::NSP;
      if (!warp_wait(fullU + 8 * sn, (kn / C::NSU) & 1, abort_flag, a.spin)) { ok = false; break; }
      q[2 * R] = U4[sn * (C::UFL / 4) + cidx];
      if (C::IMG) qi[2 * R] = I4[sn * (C::UFL / 4) + cidx];
      if (!warp_wait(fullP + 8 * sp, (kq / C::NSP) & 1, abort_flag, a.spin)) { ok = false; break; }
      float v[12], s4[4], vi[12], si4[4];
      star4<R, RW>(U4 + sc * (C::UFL / 4), q, cidx, a.W, v, s4);
      if (C::IMG) star4<R, RW>(I4 + sc * (C::UFL / 4), qi, cidx, a.W, vi, si4);
      const float4 c1 = reinterpret_cast<const float4*>(sP1 + sp * C::PFL)[ty * (BX / 4) + tx];
      const float4 c2 = reinterpret_cast<const float4*>(sP2 + sp * C::PFL)[ty * (BX / 4) + tx];
      const float4 g4 = C::IMG ? reinterpret_cast<const float4*>(sG + sp * C::PFL)[ty * (BX / 4) + tx] : c1;
      float res[4], inc[4], gnew[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const float c = v[4 + p];
        // damping of the absorbing layer (0 outside it: the undamped expressions)
        const float ad = (DAMP && MODE != MODE_IMAGE) ? sponge_a(a.L, a.W, sg.z0 + j, y, x + p) : 0.f;
        if (MODE == MODE_STEP || MODE == MODE_STEP_IMG) {
          res[p] = ad == 0.f ? fmaf(comp(c2, p), s4[p], 2.0f * c - comp(c1, p))
                             : fmaf(comp(c2, p), s4[p], 2.0f * c - (1.0f - ad) * comp(c1, p)) / (1.0f + ad);
        } else if (MODE == MODE_INC) {
          inc[p] = ad == 0.f ? fmaf(comp(c2, p), s4[p], comp(c1, p))
                             : fmaf(comp(c2, p), s4[p], (1.0f - ad) * comp(c1, p)) / (1.0f + ad);
          res[p] = c + inc[p];
        } else {
          res[p] = fmaf(comp(c1, p), s4[p], comp(c2, p));
        }
        // imaging: the step's own source field (centre) times S of the imaged field
        if (C::IMG) gnew[p] = fmaf(c, si4[p], comp(g4, p));
      }
      __syncwarp();
      if (lane == 0) {
        bar_arrive(emptyU + 8 * sc);
        bar_arrive(emptyP + 8 * sp);
      }
      if (y < a.L.ny && x < a.L.nx) {
        const long long o = a.L.off(sg.z0 + j, y, x);
        if (x + 3 < a.L.nx) {
          *reinterpret_cast<float4*>(out + o) = make_float4(res[0], res[1], res[2], res[3]);
          if (MODE == MODE_INC) *reinterpret_cast<float4*>(out2 + o) = make_float4(inc[0], inc[1], inc[2], inc[3]);
          if (C::IMG) *reinterpret_cast<float4*>(gout + o) = make_float4(gnew[0], gnew[1], gnew[2], gnew[3]);
        } else {
#pragma unroll
          for (int p = 0; p < 4; ++p)
            if (x + p < a.L.nx) {
              out[o + p] = res[p];
              if (MODE == MODE_INC) out2[o + p] = inc[p];
              if (C::IMG) gout[o + p] = gnew[p];
            }
        }
      }
#pragma unroll
      for (int k = 0; k < 2 * R; ++k) {
        q[k] = q[k + 1];
        if (C::IMG) qi[k] = qi[k + 1];
      }
    }
    if (!ok) break;
    // the last R planes were only queue heads: release them
    for (int k = nzs + R; k < nzs + 2 * R; ++k) {
      __syncwarp();
      if (lane == 0) bar_arrive(emptyU + 8 * ((ku + k) % C::NSU));
    }
    ku += nzs + 2 * R;
    kp += nzs;
  }
  if (!ok && lane == 0) atomicOr(a.err, 1);
}

// ------------------------------------------------------------------ host side
typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                             const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                             CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encode_fn() {
  static EncodeFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeFn>(p);
  });
  return fn;
}

struct MapKey {
  const void* base;
  long long nfields;
  int esize, b0, b1, b3;
  long long field;
  int px, py, pz;
  bool operator==(const MapKey& o) const {
    return base == o.base && nfields == o.nfields && esize == o.esize && b0 == o.b0 && b1 == o.b1 && b3 == o.b3 &&
           field == o.field && px == o.px && py == o.py && pz == o.pz;
  }
};

bool get_map(const Layout& L, const FieldRef& f, int bw, int bh, CUtensorMap* out) {
  return encode_field_map(L, f.base, f.nfields, 4, bw, bh, 1, out);
}

}  // namespace

// 4-D map over a family of padded fields, dims (px, py, pz, nfields), with a
// small cache of encoded maps (the buffers of one call are few and stable).
bool encode_field_map(const Layout& L, const void* base, long long nfields, int esize, int box_x, int box_y,
                      int box_fields, CUtensorMap* out) {
  static std::mutex m;
  static std::vector<std::pair<MapKey, CUtensorMap>> cache;
  const MapKey key{base, nfields, esize, box_x, box_y, box_fields, L.field, L.px, L.py, L.pz};
  std::lock_guard<std::mutex> lk(m);
  for (auto& e : cache)
    if (e.first == key) {
      *out = e.second;
      return true;
    }
  EncodeFn enc = encode_fn();
  if (!enc) return false;
  CUtensorMap map;
  const cuuint64_t es = (cuuint64_t)esize;
  const cuuint64_t dims[4] = {(cuuint64_t)L.px, (cuuint64_t)L.py, (cuuint64_t)L.pz, (cuuint64_t)nfields};
  const cuuint64_t strides[3] = {(cuuint64_t)L.px * es, (cuuint64_t)L.plane * es, (cuuint64_t)L.field * es};
  const cuuint32_t box[4] = {(cuuint32_t)box_x, (cuuint32_t)box_y, 1, (cuuint32_t)box_fields};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = enc(&map, esize == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4,
                   const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return false;
  if (cache.size() >= 64) cache.erase(cache.begin());
  cache.emplace_back(key, map);
  *out = map;
  return true;
}

namespace {

template <int R, int MODE, class C, bool DAMP>
cudaError_t launch_k(const CUtensorMap& mU, const CUtensorMap& m1, const CUtensorMap& m2, const CUtensorMap& mI,
                     const CUtensorMap& mG, const TmaArgs& t, long long blocks, cudaStream_t s) {
  const cudaError_t e = smem_limit_once<sweep3d_tma<R, MODE, C, DAMP>>((int)C::SMEM);
  if (e != cudaSuccess) return e;
  sweep3d_tma<R, MODE, C, DAMP><<<(unsigned)blocks, C::NTHREADS, C::SMEM, s>>>(mU, m1, m2, mI, mG, t);
  return cudaGetLastError();
}

template <int R, int MODE, class C>
cudaError_t launch_c(const Layout& L, const Weights& W, const StencilArgs& a, cudaStream_t s, int* err) {
  constexpr int BX = C::BX, BY = C::BY;
  CUtensorMap mU, m1, m2, mI, mG;
  if (!get_map(L, a.src, C::UW, C::UH, &mU) || !get_map(L, a.p1, BX, BY, &m1) || !get_map(L, a.p2, BX, BY, &m2))
    return cudaErrorInvalidValue;
  if (C::IMG) {
    if (!a.gout || !get_map(L, a.img, C::UW, C::UH, &mI) || !get_map(L, a.gin, BX, BY, &mG))
      return cudaErrorInvalidValue;
  } else {
    mI = mU;  // unused
    mG = m1;
  }
  TmaArgs t;
  t.L = L;
  t.W = W;
  t.f_src = a.src.f0; t.fs_src = a.src.fs;
  t.f_p1 = a.p1.f0; t.fs_p1 = a.p1.fs;
  t.f_p2 = a.p2.f0; t.fs_p2 = a.p2.fs;
  t.out = a.out;
  t.out_ss = a.out_ss;
  t.out2 = a.out2;
  t.out2_ss = a.out2_ss;
  t.f_img = a.img.f0; t.fs_img = a.img.fs;
  t.f_g = a.gin.f0; t.fs_g = a.gin.fs;
  t.gout = a.gout;
  t.gout_ss = a.gout_ss;
  t.nshots = a.nshots;
  t.ntx = (L.nx + BX - 1) / BX;
  t.nty = (L.ny + BY - 1) / BY;
  t.err = err;
  t.spin = wait_limit_cycles();
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // z chunks per tile column: the fewest that fill the CTA slots (2 per SM)
  // to at least 90 % over whole waves, else as many as keep one wave busy
  // (256^3: 64 columns x 9 chunks on 304 slots ran 3 % faster than 4 chunks,
  // which left 48 slots idle)
  const int occ = (int)std::max<size_t>(1, std::min<size_t>(2, (228 * 1024) / (C::SMEM + 1024)));
  const long long cols = (long long)t.ntx * t.nty * a.nshots, slots = (long long)occ * sms;
  const int zmax = std::max(1, L.nz / (3 * R));
  t.nzc = (int)std::max<long long>(1, std::min<long long>(slots / cols, std::max(1, L.nz / (4 * R))));
  for (int c = (int)std::max<long long>(1, (slots + cols - 1) / cols); c <= zmax; ++c) {
    const long long items = cols * c, waves = (items + slots - 1) / slots;
    if (items * 10 >= waves * slots * 9 && waves <= 3) {
      t.nzc = c;
      break;
    }
  }
  t.zchunk = (L.nz + t.nzc - 1) / t.nzc;
  t.nzc = (L.nz + t.zchunk - 1) / t.zchunk;
  t.items = cols * t.nzc;
  const long long blocks = std::min<long long>(t.items, slots);
  if (MODE != MODE_IMAGE && W.sw > 0) return launch_k<R, MODE, C, true>(mU, m1, m2, mI, mG, t, blocks, s);
  return launch_k<R, MODE, C, false>(mU, m1, m2, mI, mG, t, blocks, s);
}

// 64 x 16 tiles, 3 planes of lookahead: 128 x 8, 32 x 32 tiles measured the
// same on GB300, 4 planes the same, and one CTA per SM with 6 or 9 planes of
// lookahead 20 % slower: the consumers' per-SM throughput, not the depth of
// the copy pipeline, sets the pace.
template <int R, int MODE>
cudaError_t launch_t(const Layout& L, const Weights& W, const StencilArgs& a, cudaStream_t s, int* err) {
  if constexpr (MODE == MODE_STEP_IMG) return launch_c<R, MODE, Cfg<R, 64, 16, IMG_LA, true>>(L, W, a, s, err);
  else return launch_c<R, MODE, Cfg<R, 64, 16, 3>>(L, W, a, s, err);
}

}  // namespace

cudaError_t launch_sweep3d_tma(int mode, const Layout& L, const Weights& W, const StencilArgs& a, cudaStream_t s,
                               int* err) {
  if (W.R == 4) {
    if (mode == MODE_STEP) return launch_t<4, MODE_STEP>(L, W, a, s, err);
    if (mode == MODE_INC) return launch_t<4, MODE_INC>(L, W, a, s, err);
    if (mode == MODE_STEP_IMG) return launch_t<4, MODE_STEP_IMG>(L, W, a, s, err);
    return launch_t<4, MODE_IMAGE>(L, W, a, s, err);
  }
  if (mode == MODE_STEP) return launch_t<2, MODE_STEP>(L, W, a, s, err);
  if (mode == MODE_INC) return launch_t<2, MODE_INC>(L, W, a, s, err);
  if (mode == MODE_STEP_IMG) return launch_t<2, MODE_STEP_IMG>(L, W, a, s, err);
  return launch_t<2, MODE_IMAGE>(L, W, a, s, err);
}

}  // namespace tp
