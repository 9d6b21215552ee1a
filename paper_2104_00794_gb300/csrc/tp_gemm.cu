// Windowed probe GEMM on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// Algorithm 1 accumulates, at every time level k, ubar[x,:] += Q[k,:] * w_k[x]
// (lines 2 and 6).  Over a window of T levels this is the dense contraction
//     P[x, i] += sum_{k in window} W[x, k] * Q[k, i],
// M = grid points (10^4 .. 2*10^7), K = T (32/64), N = r (4..256), with W the
// T ring snapshots that the stencil sweeps already wrote.  Per CTA tile of 128
// points:
//   1. 128 threads load the tile's T snapshot values (coalesced rows of 128
//      points per level), split each fp32 value into tf32 hi + lo parts and
//      store both into shared memory in the K-major, no-swizzle core-matrix
//      layout (8 rows x 16 B core matrices);
//   2. one thread issues tcgen05.mma kind::tf32 (M=128, N=round16(r), K=8 per
//      instruction): hi*Qhi + lo*Qhi (+ hi*Qlo for probes that are not exact
//      in tf32), accumulating in TMEM;
//   3. tcgen05.commit arrives on an mbarrier; all warps wait (bounded), read
//      their 32 TMEM lanes with tcgen05.ld and add the tile into P in HBM.
// The hi/lo split keeps ~22 significant bits of the snapshots, so the product
// is accurate to a few 1e-7 relative; Rademacher / identity probes are exact
// in tf32 and skip the third MMA.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "tp_internal.h"

namespace tp {

namespace {

constexpr int TILE_M = 128;
constexpr long long WAIT_CYCLES = 4000000000LL;  // ~2 s at 2 GHz: bounded spin

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ float tf32_hi(float x) {
  return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
}

// Shared-memory matrix descriptor (tcgen05): start address, leading-dimension
// byte offset (between K-adjacent core matrices), stride-dimension byte offset
// (between M/N-adjacent 8-row groups), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor, kind::tf32: D f32, A and B tf32, both K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase) {
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(phase)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > WAIT_CYCLES) return false;
  }
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// Byte offset of element (row, k) in a K-major no-swizzle operand with KP
// columns: core matrix (row/8, k/4) at ((row/8)*(KP/4) + k/4)*128, row%8 at
// 16 B steps, k%4 at 4 B steps.  => LBO = 128 B, SBO = KP*32 B.
__device__ __forceinline__ uint32_t kmaj_off(int row, int k, int KP) {
  return (uint32_t)((((row >> 3) * (KP >> 2) + (k >> 2)) << 7) + ((row & 7) << 4) + ((k & 3) << 2));
}

// KP: padded window length (K); PC: probe columns whose old accumulator
// values are prefetched in registers together with the snapshots (r <= PC),
// 0 selects the chunked epilogue for large r.
template <int KP, int PC>
__global__ void __launch_bounds__(TILE_M)
probe_gemm_tf32(GemmArgs a, int NP, int ncols, long long ntiles) {
  extern __shared__ __align__(1024) unsigned char smem[];
  // layout: A_hi | A_lo | B_hi | B_lo | mbarrier | tmem slot
  const uint32_t a_bytes = TILE_M * KP * 4, b_bytes = (uint32_t)NP * KP * 4;
  unsigned char* A_hi = smem;
  unsigned char* A_lo = smem + a_bytes;
  unsigned char* B_hi = smem + 2 * a_bytes;
  unsigned char* B_lo = B_hi + b_bytes;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(B_lo + b_bytes);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 1);

  const int tid = threadIdx.x, warp = tid >> 5;
  const int shot = blockIdx.y;
  const float* ring = a.ring + shot * a.ring_ss;
  const float* Q = a.Q + shot * a.q_ss;
  float* P = static_cast<float*>(a.P) + shot * a.p_ss;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  // B operand (probe block), once per CTA: B[n][k] = Q[level0 + k + qshift][n]
  for (int e = tid; e < NP * KP; e += TILE_M) {
    const int n = e / KP, k = e % KP;
    const int row = a.level0 + k + a.qshift;
    float v = 0.f;
    if (n < a.r && k < a.nlev && row >= a.qlo && row <= a.qhi) v = Q[(long long)row * a.r + n];
    const float hi = tf32_hi(v);
    *reinterpret_cast<float*>(B_hi + kmaj_off(n, k, KP)) = hi;
    *reinterpret_cast<float*>(B_lo + kmaj_off(n, k, KP)) = v - hi;
  }
  // ring slot of the window's first level; the window (<= KP < nslots
  // levels) wraps around the ring at most once
  const int slot0 = a.level0 % a.nslots;
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  const uint32_t idesc = idesc_tf32(TILE_M, NP);
  const uint32_t sbo = KP * 32, lbo = 128;
  const uint32_t a_hi_u = smem_u32(A_hi), a_lo_u = smem_u32(A_lo);
  const uint32_t b_hi_u = smem_u32(B_hi), b_lo_u = smem_u32(B_lo);
  const uint32_t bar = smem_u32(mbar);
  bool ok = true;
  uint32_t phase = 0;

  // register prefetch of one tile: the snapshots (A) and the old accumulators
  float av[KP];
  float pv[PC > 0 ? PC : 1];
  // tile -> (grid row, 128-point segment) -> padded offset of its first point
  const int nxt = (a.L.nx + TILE_M - 1) / TILE_M;
  auto tile_base = [&](long long tile) -> long long {
    const long long row = tile / nxt;
    const int xb = (int)(tile % nxt);
    return a.L.off(row / a.L.ny, row % a.L.ny, (long long)xb * TILE_M);
  };
  auto load_tile = [&](long long tile) {
    const long long pt = tile_base(tile) + tid;
    const bool in = true;
#pragma unroll
    for (int k = 0; k < KP; ++k) {
      const int sl = slot0 + k >= a.nslots ? slot0 + k - a.nslots : slot0 + k;
      av[k] = (in && k < a.nlev) ? __ldcs(ring + (long long)sl * a.slot_stride + pt) : 0.f;
    }
#pragma unroll
    for (int i = 0; i < PC; ++i) pv[i] = (in && i < a.r) ? __ldcs(P + (long long)i * a.pstride + pt) : 0.f;
  };
  if ((long long)blockIdx.x < ntiles) load_tile(blockIdx.x);

  for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    const long long m0 = tile_base(tile);
    // 1. split the snapshots into tf32 hi + lo and stage them K-major
#pragma unroll
    for (int k4 = 0; k4 < KP; k4 += 4) {
      float4 hi, lo;
      hi.x = tf32_hi(av[k4 + 0]); hi.y = tf32_hi(av[k4 + 1]); hi.z = tf32_hi(av[k4 + 2]); hi.w = tf32_hi(av[k4 + 3]);
      lo.x = av[k4 + 0] - hi.x; lo.y = av[k4 + 1] - hi.y; lo.z = av[k4 + 2] - hi.z; lo.w = av[k4 + 3] - hi.w;
      const uint32_t o = kmaj_off(tid, k4, KP);
      *reinterpret_cast<float4*>(A_hi + o) = hi;
      *reinterpret_cast<float4*>(A_lo + o) = lo;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    // 2. one thread issues the MMAs
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int kk = 0; kk < KP / 8; ++kk) {
        const uint32_t ko = kk * 2 * 128;  // two 16-byte K chunks per MMA
        const uint64_t ah = smem_desc(a_hi_u + ko, lbo, sbo), al = smem_desc(a_lo_u + ko, lbo, sbo);
        const uint64_t bh = smem_desc(b_hi_u + ko, lbo, sbo), bl = smem_desc(b_lo_u + ko, lbo, sbo);
        mma_tf32(tmem, ah, bh, idesc, kk > 0 ? 1u : 0u);
        mma_tf32(tmem, al, bh, idesc, 1u);
        if (a.q_has_lo) mma_tf32(tmem, ah, bl, idesc, 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                   : "memory");
    }
    __syncwarp();
    // 3. while the tensor cores run, fetch the next tile
    float pc[PC > 0 ? PC : 1];
#pragma unroll
    for (int i = 0; i < PC; ++i) pc[i] = pv[i];
    if (tile + gridDim.x < ntiles) load_tile(tile + gridDim.x);
    // 4. epilogue: TMEM lanes 32*warp.. -> P (coalesced per probe column)
    // one thread polls the barrier; the others wait at the CTA barrier
    const int all_done = __syncthreads_and(tid == 0 ? (mbar_wait(bar, phase) ? 1 : 0) : 1);
    if (!all_done) {
      ok = false;
      if (tid == 0) atomicExch(a.err, 1);
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
      const long long prow = m0 + warp * 32 + (tid & 31);  // padded offset of this lane's point
      const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
      if (PC > 0) {
#pragma unroll
        for (int c = 0; c < (PC > 0 ? PC / 16 : 1); ++c) {
          if (c * 16 < NP) {  // uniform
            float acc[16];
            tmem_ld16(trow + (uint32_t)(c * 16), acc);
            {
#pragma unroll
              for (int j = 0; j < 16; ++j)
                if (c * 16 + j < a.r) P[(long long)(c * 16 + j) * a.pstride + prow] = pc[c * 16 + j] + acc[j];
            }
          }
        }
      } else {
        for (int c0 = 0; c0 < NP; c0 += 16) {
          float acc[16];
          tmem_ld16(trow + (uint32_t)c0, acc);
          {
            float old[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) old[j] = (c0 + j < a.r) ? P[(long long)(c0 + j) * a.pstride + prow] : 0.f;
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (c0 + j < a.r) P[(long long)(c0 + j) * a.pstride + prow] = old[j] + acc[j];
          }
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
  }
}

// ------------------------------------------------------------------ TMA variant
// For r <= 32: a producer warp streams each tile's window rows (nlev x 512 B)
// and old accumulator rows (r x 512 B) into a 2-stage shared-memory ring with
// cp.async.bulk (completion counted on an mbarrier); four worker warps split
// the snapshots into tf32 hi/lo operands, one thread issues the MMAs, and the
// workers add the TMEM tile to the staged accumulators and store them.  Two
// CTAs per SM (KP = 32) keep four tiles of copies in flight per SM without
// holding them in registers.
constexpr int GNS = 2;      // stages
constexpr int GRP = 32;     // accumulator rows staged per tile (r <= 32)
constexpr int GW = 4;       // worker warps
constexpr int GTHREADS = (GW + 1) * 32;

__device__ __forceinline__ void mbar_init(uint32_t b, uint32_t n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(b), "r"(n));
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(b) : "memory");
}
__device__ __forceinline__ bool mbar_wait_abort(uint32_t bar, uint32_t phase, volatile int* abort_flag) {
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(phase)
        : "memory");
    if (done) return true;
    if (*abort_flag) return false;
    if (clock64() - t0 > WAIT_CYCLES) {
      *abort_flag = 1;
      return false;
    }
  }
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void bar_named(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }

// ACC: accumulator storage (0 fp32, 1 bf16, 2 bf16 value + bf16 compensation),
// or 3: dot mode -- the staged rows are the r forward fields ubar (fp32) and
// the gradient row, and the tile is folded into the gradient at once.
template <int KP, int ACC>
struct GCfg {
  static constexpr uint32_t PROW = (ACC == 0 || ACC == 3) ? TILE_M * 4 : TILE_M * 2;  // bytes of one staged row
  static constexpr uint32_t PBYTES = GRP * PROW * (ACC == 2 ? 2 : 1) + (ACC == 3 ? PROW : 0);
  static constexpr uint32_t STAGE = (uint32_t)KP * TILE_M * 4 + PBYTES;  // A rows then accumulator rows
  static constexpr uint32_t ABYTES = TILE_M * KP * 4;
  static constexpr uint32_t BBYTES = GRP * KP * 4;
  static constexpr size_t SMEM = (size_t)GNS * STAGE + 2 * ABYTES + 2 * BBYTES + 8 * (2 * GNS + 1) + 32;
};

template <int KP, int ACC>
__global__ void __launch_bounds__(GTHREADS)
probe_gemm_tma(GemmArgs a, int NP, long long ntiles) {
  using C = GCfg<KP, ACC>;
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* stage0 = smem;
  unsigned char* A_hi = smem + GNS * C::STAGE;
  unsigned char* A_lo = A_hi + C::ABYTES;
  unsigned char* B_hi = A_lo + C::ABYTES;
  unsigned char* B_lo = B_hi + C::BBYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(B_lo + C::BBYTES);
  const uint32_t full = smem_u32(bars), empty = full + 8 * GNS, mma_bar = empty + 8 * GNS;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * GNS + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int shot = blockIdx.y;
  const float* ring = a.ring + shot * a.ring_ss;
  const float* Q = a.Q + shot * a.q_ss;
  float* Pf = static_cast<float*>(a.P) + shot * a.p_ss;                  // ACC == 0
  __nv_bfloat16* Ph = static_cast<__nv_bfloat16*>(a.P) + shot * a.p_ss;  // ACC != 0
  const int nxt = (a.L.nx + TILE_M - 1) / TILE_M;
  auto tile_base = [&](long long tile) -> long long {
    const long long row = tile / nxt;
    return a.L.off(row / a.L.ny, row % a.L.ny, (long long)(tile % nxt) * TILE_M);
  };

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(32));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int s = 0; s < GNS; ++s) {
      mbar_init(full + 8 * s, 1);
      mbar_init(empty + 8 * s, GW);
    }
    mbar_init(mma_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // B operand (probe block) once per CTA, as in probe_gemm_tf32
  for (int e = tid; e < NP * KP; e += GTHREADS) {
    const int n = e / KP, k = e % KP;
    const int row = a.level0 + k + a.qshift;
    float v = 0.f;
    if (n < a.r && k < a.nlev && row >= a.qlo && row <= a.qhi) v = Q[(long long)row * a.r + n];
    const float hi = tf32_hi(v);
    *reinterpret_cast<float*>(B_hi + kmaj_off(n, k, KP)) = hi;
    *reinterpret_cast<float*>(B_lo + kmaj_off(n, k, KP)) = v - hi;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const int slot0 = a.level0 % a.nslots;

  if (warp == GW) {
    // ------------------------------------------------------------ producer warp
    const int ncp = ACC == 2 ? 2 * a.r : (ACC == 3 ? a.r + 1 : a.r);  // accumulator rows copied per tile
    const uint32_t bytes = (uint32_t)a.nlev * TILE_M * 4 + (uint32_t)ncp * C::PROW;
    bool ok = true;
    uint32_t it = 0;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
      const int s = it % GNS;
      if (it >= (uint32_t)GNS) {
        bool w = true;
        if (lane == 0) w = mbar_wait_abort(empty + 8 * s, ((it / GNS) - 1) & 1, abort_flag);
        if (!__shfl_sync(0xffffffffu, w ? 1 : 0, 0)) { ok = false; break; }
      }
      if (lane == 0) mbar_expect_tx(full + 8 * s, bytes);
      __syncwarp();
      const long long base = tile_base(tile);
      const uint32_t dst = smem_u32(stage0 + s * C::STAGE);
      const uint32_t pdst = dst + (uint32_t)KP * TILE_M * 4;
      for (int c = lane; c < a.nlev + ncp; c += 32) {
        if (c < a.nlev) {
          const int sl = slot0 + c >= a.nslots ? slot0 + c - a.nslots : slot0 + c;
          bulk_g2s(dst + (uint32_t)c * TILE_M * 4, ring + (long long)sl * a.slot_stride + base, TILE_M * 4, full + 8 * s);
        } else {
          const int idx = c - a.nlev;
          if (ACC == 3 && idx == a.r) {  // the gradient row, staged after GRP field rows
            bulk_g2s(pdst + (uint32_t)GRP * C::PROW, a.G + shot * a.g_ss + base, C::PROW, full + 8 * s);
          } else if (ACC == 0 || ACC == 3) {
            bulk_g2s(pdst + (uint32_t)idx * C::PROW, Pf + (long long)idx * a.pstride + base, C::PROW, full + 8 * s);
          } else if (ACC == 1 || idx < a.r) {  // bf16 values
            bulk_g2s(pdst + (uint32_t)idx * C::PROW, Ph + (long long)idx * a.pstride + base, C::PROW, full + 8 * s);
          } else {                              // bf16 compensations, staged after GRP value rows
            const int i = idx - a.r;
            bulk_g2s(pdst + (uint32_t)(GRP + i) * C::PROW, Ph + (long long)(a.r + i) * a.pstride + base, C::PROW,
                     full + 8 * s);
          }
        }
      }
    }
    if (!ok && lane == 0) atomicOr(a.err, 1);
    // drain: every issued stage must have landed before the CTA exits
    if (lane == 0) {
      for (uint32_t j = (it > (uint32_t)GNS ? it - GNS : 0); j < it; ++j) {
        const long long t0 = clock64();
        while (!mbar_wait_abort(full + 8 * (j % GNS), (j / GNS) & 1, abort_flag) && clock64() - t0 < WAIT_CYCLES) {}
      }
    }
  } else {
    // ------------------------------------------------------------ workers
    const uint32_t idesc = idesc_tf32(TILE_M, NP);
    const uint32_t sbo = KP * 32, lbo = 128;
    const uint32_t a_hi_u = smem_u32(A_hi), a_lo_u = smem_u32(A_lo);
    const uint32_t b_hi_u = smem_u32(B_hi), b_lo_u = smem_u32(B_lo);
    uint32_t it = 0, mph = 0;
    bool ok = true;
    for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++it) {
      const int s = it % GNS;
      if (!mbar_wait_abort(full + 8 * s, (it / GNS) & 1, abort_flag)) { ok = false; }
      bar_named(1, GW * 32);
      if (*abort_flag) { ok = false; break; }
      const float* sA = reinterpret_cast<const float*>(stage0 + s * C::STAGE);
      const float* sP = sA + KP * TILE_M;
      const __nv_bfloat16* sPh = reinterpret_cast<const __nv_bfloat16*>(sP);
      // 1. split this thread's point column of the staged snapshots
#pragma unroll
      for (int k4 = 0; k4 < KP; k4 += 4) {
        float v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) v[j] = (k4 + j < a.nlev) ? sA[(k4 + j) * TILE_M + tid] : 0.f;
        float4 hi, lo;
        hi.x = tf32_hi(v[0]); hi.y = tf32_hi(v[1]); hi.z = tf32_hi(v[2]); hi.w = tf32_hi(v[3]);
        lo.x = v[0] - hi.x; lo.y = v[1] - hi.y; lo.z = v[2] - hi.z; lo.w = v[3] - hi.w;
        const uint32_t o = kmaj_off(tid, k4, KP);
        *reinterpret_cast<float4*>(A_hi + o) = hi;
        *reinterpret_cast<float4*>(A_lo + o) = lo;
      }
      // 2. old accumulators of this point, then release the stage
      float pold[GRP];  // old accumulators, or the forward fields in dot mode
#pragma unroll
      for (int i = 0; i < GRP; ++i) {
        float v = 0.f;
        if (i < a.r) {
          if (ACC == 0 || ACC == 3) v = sP[i * TILE_M + tid];
          else v = __bfloat162float(sPh[i * TILE_M + tid]);
          if (ACC == 2) v += __bfloat162float(sPh[(GRP + i) * TILE_M + tid]);
        }
        pold[i] = v;
      }
      const float gold = ACC == 3 ? sP[GRP * TILE_M + tid] : 0.f;
      __syncwarp();
      if (lane == 0) mbar_arrive(empty + 8 * s);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      bar_named(1, GW * 32);
      // 3. MMAs
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int kk = 0; kk < KP / 8; ++kk) {
          const uint32_t ko = kk * 2 * 128;
          const uint64_t ah = smem_desc(a_hi_u + ko, lbo, sbo), al = smem_desc(a_lo_u + ko, lbo, sbo);
          const uint64_t bh = smem_desc(b_hi_u + ko, lbo, sbo), bl = smem_desc(b_lo_u + ko, lbo, sbo);
          mma_tf32(tmem, ah, bh, idesc, kk > 0 ? 1u : 0u);
          mma_tf32(tmem, al, bh, idesc, 1u);
          if (a.q_has_lo) mma_tf32(tmem, ah, bl, idesc, 1u);
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mma_bar)
                     : "memory");
      }
      // 4. epilogue
      int done = 1;
      if (tid == 0) done = mbar_wait_abort(mma_bar, mph, abort_flag) ? 1 : 0;
      mph ^= 1u;
      bar_named(1, GW * 32);
      if (*abort_flag || !done) { ok = false; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const long long prow = tile_base(tile) + tid;
      const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
      float dot = 0.f;
#pragma unroll
      for (int c = 0; c < GRP / 16; ++c) {
        if (c * 16 < NP) {
          float acc[16];
          tmem_ld16(trow + (uint32_t)(c * 16), acc);
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int i = c * 16 + j;
            if (ACC == 3) {
              if (i < a.r) dot = fmaf(pold[i], acc[j], dot);
            } else if (i < a.r) {
              const float nv = pold[i] + acc[j];
              if (ACC == 0) {
                Pf[(long long)i * a.pstride + prow] = nv;
              } else {
                const __nv_bfloat16 hv = __float2bfloat16_rn(nv);
                Ph[(long long)i * a.pstride + prow] = hv;
                // compensation: the rounding error of the stored value
                if (ACC == 2) Ph[(long long)(a.r + i) * a.pstride + prow] = __float2bfloat16_rn(nv - __bfloat162float(hv));
              }
            }
          }
        }
      }
      if (ACC == 3) a.G[shot * a.g_ss + prow] = gold + dot;
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
    if (!ok && tid == 0) atomicOr(a.err, 1);
  }
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(32));
  }
}

template <int KP, int ACC>
cudaError_t launch_tma(const GemmArgs& a, cudaStream_t s) {
  using C = GCfg<KP, ACC>;
  const int NP = std::max(16, (a.r + 15) / 16 * 16);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(probe_gemm_tma<KP, ACC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    attr = true;
  }
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int occ = std::max(1, std::min(4, (int)((228 * 1024) / (C::SMEM + 1024))));
  const long long ntiles = (long long)a.L.nz * a.L.ny * ((a.L.nx + TILE_M - 1) / TILE_M);
  const long long grid_x = std::min<long long>(ntiles, (long long)sms * occ);
  dim3 grid((unsigned)grid_x, a.nshots);
  probe_gemm_tma<KP, ACC><<<grid, GTHREADS, C::SMEM, s>>>(a, NP, ntiles);
  return cudaGetLastError();
}

template <int KP, int PC>
cudaError_t launch_kp(const GemmArgs& a, cudaStream_t s) {
  const int NP = std::max(16, (a.r + 15) / 16 * 16);
  int ncols = 32;
  while (ncols < NP) ncols <<= 1;
  const size_t smem = (size_t)2 * TILE_M * KP * 4 + (size_t)2 * NP * KP * 4 + 16;
  static int regs = 0;
  if (regs == 0) {
    cudaFuncSetAttribute(probe_gemm_tf32<KP, PC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncAttributes fa;
    regs = cudaFuncGetAttributes(&fa, probe_gemm_tf32<KP, PC>) == cudaSuccess ? std::max(fa.numRegs, 1) : 255;
  }
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // CTAs per SM: registers, shared memory (228 KB, 1 KB reserved per CTA), TMEM columns
  const int by_regs = 65536 / (((regs + 7) / 8 * 8) * TILE_M);
  const int by_smem = (int)((228 * 1024) / (smem + 1024));
  const int by_tmem = 512 / ncols;
  const int occ = std::max(1, std::min(std::min(by_regs, by_smem), std::min(by_tmem, 8)));
  const long long ntiles = (long long)a.L.nz * a.L.ny * ((a.L.nx + TILE_M - 1) / TILE_M);
  const long long grid_x = std::min<long long>(ntiles, (long long)sms * occ);
  dim3 grid((unsigned)grid_x, a.nshots);
  probe_gemm_tf32<KP, PC><<<grid, TILE_M, smem, s>>>(a, NP, ncols, ntiles);
  return cudaGetLastError();
}

}  // namespace

int gemm_kpad(int T) { return T <= 32 ? 32 : 64; }

cudaError_t launch_probe_gemm(const GemmArgs& a, cudaStream_t s) {
  if (a.nlev <= 0) return cudaSuccess;
  prof_before(2, s);  // TP_KERNEL_PROBE_GEMM
  static const int variant = [] {  // TP_PROBE_GEMM=regs selects the register-staged kernel
    const char* e = getenv("TP_PROBE_GEMM");
    return (e && strcmp(e, "regs") == 0) ? 1 : 0;
  }();
  cudaError_t e;
  if (a.acc != 0 || (a.r <= GRP && variant == 0)) {  // bf16 storage and dot mode exist on this path only (r <= 32)
    if (a.nlev <= 32)
      e = a.acc == 0 ? launch_tma<32, 0>(a, s)
                     : (a.acc == 1 ? launch_tma<32, 1>(a, s) : (a.acc == 2 ? launch_tma<32, 2>(a, s) : launch_tma<32, 3>(a, s)));
    else
      e = a.acc == 0 ? launch_tma<64, 0>(a, s)
                     : (a.acc == 1 ? launch_tma<64, 1>(a, s) : (a.acc == 2 ? launch_tma<64, 2>(a, s) : launch_tma<64, 3>(a, s)));
  } else if (a.nlev <= 32) {
    e = a.r <= 16 ? launch_kp<32, 16>(a, s) : (a.r <= 32 ? launch_kp<32, 32>(a, s) : launch_kp<32, 0>(a, s));
  } else {
    e = a.r <= 16 ? launch_kp<64, 16>(a, s) : (a.r <= 32 ? launch_kp<64, 32>(a, s) : launch_kp<64, 0>(a, s));
  }
  prof_after(2, s);
  return e;
}

}  // namespace tp
