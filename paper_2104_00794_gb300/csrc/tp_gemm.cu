// Windowed probe GEMM on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// Algorithm 1 accumulates, at every time level k, ubar[x,:] += Q[k,:] * w_k[x]
// (lines 2 and 6).  Over a window of T levels this is the dense contraction
//     P[x, i] += sum_{k in window} W[x, k] * Q[k, i],
// M = grid points (10^4 .. 2*10^7), K = T (32/64/128), N = r (4..256), with W the
// T ring snapshots that the stencil sweeps already wrote.  Every tile of 128
// points splits its fp32 snapshots into tf32 hi + lo parts in shared memory
// (K-major, no-swizzle core-matrix layout: 8 rows x 16 B core matrices), one
// thread issues tcgen05.mma kind::tf32 (M=128, N=round16(r), K=8 per
// instruction: hi*Qhi + lo*Qhi, + hi*Qlo for probes that are not exact in
// tf32) into TMEM, and the tile is read back with tcgen05.ld and added to P.
// The hi/lo split keeps ~22 significant bits of the snapshots, so the product
// is accurate to a few 1e-7 relative; Rademacher / identity probes are exact
// in tf32 and skip the third MMA.
//
// Two kernels:
//   * probe_gemm_ws (r <= 32, every accumulator storage and the dot mode of
//     the single-accumulator adjoint): a warp-specialised pipeline with 4-D
//     TMA tensor copies and stores, one CTA per SM (the SMs shared among the
//     shots of a batch); described where it is defined below.  It runs at the
//     HBM roofline.
//   * probe_gemm_tf32 (r > 32, e.g. identity probes with r = nt in tests):
//     128 threads per tile load the snapshots through registers, one thread
//     issues the MMAs, all threads drain TMEM into P.
#include <cuda_bf16.h>

#include <algorithm>

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

// ------------------------------------------------------------ pipelined variant
// For r <= 32 (every accumulator kind and the dot mode) the window GEMM runs
// as a warp-specialised pipeline, one CTA per SM looping over 128-point tiles:
//   warp 0      producer of the window rows: per tile one or two 4-D TMA
//               tensor copies (nlev x 512 B; two where the ring wraps) into
//               NSR snapshot stages;
//   warp 10     producer of the old accumulator rows (and, in dot mode, the
//               gradient row): one or two TMA copies into NSA stages;
//   warp 1      allocates TMEM; one lane issues the tcgen05 MMAs of tile k
//               into TMEM buffer k % 2 and commits them to mdone[k % 2];
//   warps 2-5   converters: split tile k's snapshots into tf32 hi/lo operand
//               buffers (NA of them) in the K-major core-matrix layout;
//   warps 6-9   epilogue: read tile k's accumulator rows from the stage, wait
//               for mdone, add the TMEM tile and store (or, in dot mode, fold
//               it into the gradient row).
// Tiles k+1 (convert), k (MMA) and k-1 (epilogue) overlap, and the stages
// keep copies of later tiles in flight.  A few large tensor copies per tile
// instead of one bulk copy per 512-B row: issuing ~65 row copies per tile
// from one warp capped a CTA at about one tile per 2.8 us.  Every wait is
// bounded: a timeout sets a shared abort flag that every role checks, so all
// roles leave their loops.
constexpr int GRP = 32;          // accumulator rows staged per tile (r <= 32)
constexpr int WS_THREADS = 352;  // eleven warps
constexpr int WS_TMEM_COLS = 64; // two accumulator buffers of 32 columns

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
__device__ __forceinline__ void tma_store_rows(const CUtensorMap* map, int c0, int c1, int c2, int c3, uint32_t src) {
  asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3, %4}], [%5];"
               ::"l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(src)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_read_all_but_one() {
  asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// named barrier that also ORs a predicate over the participating threads, so
// that every thread takes the same abort decision
__device__ __forceinline__ bool bar_or(int id, int n, bool pred) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, %2, %3, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)pred), "r"(id), "r"(n)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void tma_rows(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                         uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}

// ACC: accumulator storage (0 fp32, 1 bf16, 2 bf16 value + bf16 compensation),
// or 3: dot mode -- the staged rows are the r forward fields ubar (fp32) and
// the gradient row, and the tile is folded into the gradient at once.
// KP: the window's K extent (32, 64 or 128).  Snapshots move and are split
// in sub-tiles of KS = 32 levels (one stage, one operand buffer each); a
// longer window is several sub-tiles whose MMAs accumulate into the same
// TMEM tile.
constexpr int KS = 32;
constexpr int MAXSUB = 4;

template <int KP, int ACC>
struct WCfg {
  static constexpr int NSR = 4;                 // snapshot stages (one sub-tile each)
  static constexpr int NSA = KP == 32 ? 5 : (KP == 64 ? 4 : 3);  // accumulator stages
  static constexpr int NA = 2;                  // operand buffers (hi + lo each)
  static constexpr uint32_t RSTAGE = (uint32_t)KS * TILE_M * 4;
  static constexpr uint32_t PROW = (ACC == 0 || ACC == 3) ? TILE_M * 4 : TILE_M * 2;  // one staged row
  static constexpr uint32_t ASTAGE = GRP * PROW * (ACC == 2 ? 2 : 1) + (ACC == 3 ? PROW : 0);
  static constexpr uint32_t ABYTES = TILE_M * KS * 4;
  static constexpr uint32_t BBYTES = GRP * KP * 4;
  // barriers: full_r, empty_r [NSR]; full_a, empty_a [NSA]; aready, afree [NA]; mdone, tfree [2]
  static constexpr int NBAR = 2 * NSR + 2 * NSA + 2 * NA + 4;
  static constexpr size_t SMEM =
      (size_t)NSR * RSTAGE + (size_t)NSA * ASTAGE + (size_t)NA * 2 * ABYTES + 2 * BBYTES + 8 * NBAR + 16;
};

// The window's sub-tiles: rows (levels) of each, the ring slot of its first
// level and the rows before the ring wraps.
struct SubTiles {
  int nsub;
  int rows[MAXSUB], slot[MAXSUB], n1[MAXSUB];
};

// mRj0 / mRj1: the ring (all shots' slots as one field family) with
// boxes of sub-tile j's rows before and after the ring wraps; mA: the
// accumulator family (box: the rows of one shot); mG: the gradient family of
// the dot mode (box: one row).
template <int KP, int ACC>
__global__ void __launch_bounds__(WS_THREADS, 1)
probe_gemm_ws(const __grid_constant__ CUtensorMap mR00, const __grid_constant__ CUtensorMap mR01,
              const __grid_constant__ CUtensorMap mR10, const __grid_constant__ CUtensorMap mR11,
              const __grid_constant__ CUtensorMap mR20, const __grid_constant__ CUtensorMap mR21,
              const __grid_constant__ CUtensorMap mR30, const __grid_constant__ CUtensorMap mR31,
              const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mG, GemmArgs a, int NP,
              long long ntiles, SubTiles st_) {
  using C = WCfg<KP, ACC>;
  constexpr int NSR = C::NSR, NSA = C::NSA, NA = C::NA;
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* rstage0 = smem;
  unsigned char* astage0 = rstage0 + NSR * C::RSTAGE;
  unsigned char* A0 = astage0 + NSA * C::ASTAGE;  // operand buffer j: hi at A0 + 2j*ABYTES, lo after it
  unsigned char* B_hi = A0 + NA * 2 * C::ABYTES;
  unsigned char* B_lo = B_hi + C::BBYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(B_lo + C::BBYTES);
  const uint32_t full_r = smem_u32(bars), empty_r = full_r + 8 * NSR;
  const uint32_t full_a = empty_r + 8 * NSR, empty_a = full_a + 8 * NSA;
  const uint32_t aready = empty_a + 8 * NSA, afree = aready + 8 * NA, mdone = afree + 8 * NA, tfree = mdone + 16;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + C::NBAR);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int shot = blockIdx.y;
  const int nxt = (a.L.nx + TILE_M - 1) / TILE_M;
  auto tile_base = [&](long long tile) -> long long {
    const long long row = tile / nxt;
    return a.L.off(row / a.L.ny, row % a.L.ny, (long long)(tile % nxt) * TILE_M);
  };

  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(WS_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int s = 0; s < NSR; ++s) {
      mbar_init(full_r + 8 * s, 1);
      mbar_init(empty_r + 8 * s, TILE_M);
    }
    for (int s = 0; s < NSA; ++s) {
      mbar_init(full_a + 8 * s, 1);
      mbar_init(empty_a + 8 * s, ACC == 3 ? TILE_M : 1);
    }
    for (int j = 0; j < NA; ++j) {
      mbar_init(aready + 8 * j, TILE_M);
      mbar_init(afree + 8 * j, 1);
    }
    for (int j = 0; j < 2; ++j) {
      mbar_init(mdone + 8 * j, 1);
      mbar_init(tfree + 8 * j, ACC == 3 ? TILE_M : 1);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // B operand (the window's probe block, shared by every tile), tf32 hi/lo
  const float* Q = a.Q + shot * a.q_ss;
  for (int e = tid; e < NP * KP; e += WS_THREADS) {
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

  const int cy = a.L.ndim == 3 ? H : 0;
  // sub-tile fields by value (no dynamic indexing, which would go through local memory)
  const int nsub = st_.nsub;
  auto pick = [](int j, int v0, int v1, int v2, int v3) { return j == 0 ? v0 : (j == 1 ? v1 : (j == 2 ? v2 : v3)); };
  auto sub_rows = [&](int j) { return pick(j, st_.rows[0], st_.rows[1], st_.rows[2], st_.rows[3]); };
  auto sub_slot = [&](int j) { return pick(j, st_.slot[0], st_.slot[1], st_.slot[2], st_.slot[3]); };
  auto sub_n1 = [&](int j) { return pick(j, st_.n1[0], st_.n1[1], st_.n1[2], st_.n1[3]); };
  if (warp == 0 || warp == 10) {
    // ------------------------------------------------------------ producers (lane 0 issues):
    // warp 0 the snapshot rows (one stage per sub-tile), warp 10 the
    // accumulator rows (and the gradient row)
    const bool snap = warp == 0;
    const int NS = snap ? NSR : NSA;
    const uint32_t full = snap ? full_r : full_a, empty = snap ? empty_r : empty_a;
    const int nacc = ACC == 2 ? 2 * a.r : a.r;  // accumulator rows of one shot
    const int nper = snap ? nsub : 1;           // stages per tile
    bool ok = true;
    uint32_t k = 0;  // stages issued
    for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
      const long long row = tile / nxt;
      const int c0 = HX + (int)(tile % nxt) * TILE_M, c1 = (int)(row % a.L.ny) + cy, c2 = (int)(row / a.L.ny) + H;
      for (int j = 0; j < nper; ++j, ++k) {
        const int st = k % NS;
        if (k >= (uint32_t)NS) {
          bool w = true;
          if (lane == 0) w = mbar_wait_abort(empty + 8 * st, ((k / NS) - 1) & 1, abort_flag);
          if (!__shfl_sync(0xffffffffu, w ? 1 : 0, 0)) { ok = false; break; }
        }
        if (lane == 0) {
          if (snap) {
            mbar_expect_tx(full + 8 * st, (uint32_t)sub_rows(j) * TILE_M * 4);
            const uint32_t dst = smem_u32(rstage0 + st * C::RSTAGE);
            const CUtensorMap* m0 = j == 0 ? &mR00 : (j == 1 ? &mR10 : (j == 2 ? &mR20 : &mR30));
            const CUtensorMap* m1 = j == 0 ? &mR01 : (j == 1 ? &mR11 : (j == 2 ? &mR21 : &mR31));
            tma_rows(dst, m0, c0, c1, c2, shot * a.nslots + sub_slot(j), full + 8 * st);
            if (sub_n1(j) < sub_rows(j))
              tma_rows(dst + (uint32_t)sub_n1(j) * TILE_M * 4, m1, c0, c1, c2, shot * a.nslots, full + 8 * st);
          } else {
            mbar_expect_tx(full + 8 * st, (uint32_t)nacc * C::PROW + (ACC == 3 ? C::PROW : 0));
            const uint32_t dst = smem_u32(astage0 + st * C::ASTAGE);
            tma_rows(dst, &mA, c0, c1, c2, shot * nacc, full + 8 * st);
            if (ACC == 3) tma_rows(dst + (uint32_t)GRP * C::PROW, &mG, c0, c1, c2, shot, full + 8 * st);
          }
        }
        __syncwarp();
      }
    }
    if (!ok && lane == 0) atomicOr(a.err, 1);
    // every issued copy must have landed before the CTA exits (bounded waits)
    if (lane == 0) {
      for (uint32_t j = (k > (uint32_t)NS ? k - NS : 0); j < k; ++j) {
        const long long t0 = clock64();
        while (!mbar_wait_abort(full + 8 * (j % NS), (j / NS) & 1, abort_flag) && clock64() - t0 < WAIT_CYCLES) {}
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc = idesc_tf32(TILE_M, NP);
      const uint32_t sbo_a = KS * 32, sbo_b = KP * 32, lbo = 128;
      const uint32_t b_hi_u = smem_u32(B_hi), b_lo_u = smem_u32(B_lo);
      bool ok = true;
      long long committed = -1;  // last sub-tile whose MMAs were committed to afree
      uint32_t k = 0, kc = 0;
      for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++k) {
        const int jt = k & 1;
        if (k >= 2 && !mbar_wait_abort(tfree + 8 * jt, ((k - 2) / 2) & 1, abort_flag)) { ok = false; break; }
        const uint32_t d = tmem + (uint32_t)(jt * 32);
        for (int j = 0; j < nsub; ++j, ++kc) {
          const int ja = kc % NA;
          if (!mbar_wait_abort(aready + 8 * ja, (kc / NA) & 1, abort_flag)) { ok = false; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t a_hi_u = smem_u32(A0 + 2 * ja * C::ABYTES), a_lo_u = a_hi_u + C::ABYTES;
          const uint32_t bo = (uint32_t)j * (KS / 4) * 128;  // sub-tile j's K columns in the K = KP layout of B
#pragma unroll
          for (int kk = 0; kk < KS / 8; ++kk) {
            const uint32_t ko = kk * 2 * 128;
            const uint64_t ah = smem_desc(a_hi_u + ko, lbo, sbo_a), al = smem_desc(a_lo_u + ko, lbo, sbo_a);
            const uint64_t bh = smem_desc(b_hi_u + bo + ko, lbo, sbo_b), bl = smem_desc(b_lo_u + bo + ko, lbo, sbo_b);
            mma_tf32(d, ah, bh, idesc, (j > 0 || kk > 0) ? 1u : 0u);
            mma_tf32(d, al, bh, idesc, 1u);
            if (a.q_has_lo) mma_tf32(d, ah, bl, idesc, 1u);
          }
          // operand buffer ja is free once these MMAs have read it
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(afree + 8 * ja)
                       : "memory");
          committed = kc;
        }
        if (!ok) break;
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mdone + 8 * jt)
                     : "memory");
      }
      if (!ok) {
        atomicOr(a.err, 1);
        // let the MMAs already issued finish before TMEM is released (bounded)
        if (committed >= 0) {
          const uint32_t kl = (uint32_t)committed;
          mbar_wait(afree + 8 * (kl % NA), (kl / NA) & 1);
        }
      }
    }
    __syncwarp();
  } else if (warp < 6) {
    // ------------------------------------------------------------ converters: one point per thread
    const int m = tid - 64;
    bool ok = true;
    uint32_t kc = 0;  // sub-tiles converted
    for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
      for (int j = 0; j < nsub; ++j, ++kc) {
        const int sr = kc % NSR, ja = kc % NA;
        if (!mbar_wait_abort(full_r + 8 * sr, (kc / NSR) & 1, abort_flag)) { ok = false; break; }
        if (kc >= (uint32_t)NA) {  // the MMAs of sub-tile kc - NA have finished reading operand buffer ja
          const uint32_t kp = kc - NA;
          if (!mbar_wait_abort(afree + 8 * ja, (kp / NA) & 1, abort_flag)) { ok = false; break; }
        }
        const float* sA = reinterpret_cast<const float*>(rstage0 + sr * C::RSTAGE);
        unsigned char* A_hi = A0 + 2 * ja * C::ABYTES;
        unsigned char* A_lo = A_hi + C::ABYTES;
        const int rows = sub_rows(j);
#pragma unroll
        for (int k4 = 0; k4 < KS; k4 += 4) {
          float v[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) v[q] = (k4 + q < rows) ? sA[(k4 + q) * TILE_M + m] : 0.f;
          float4 hi, lo;
          hi.x = tf32_hi(v[0]); hi.y = tf32_hi(v[1]); hi.z = tf32_hi(v[2]); hi.w = tf32_hi(v[3]);
          lo.x = v[0] - hi.x; lo.y = v[1] - hi.y; lo.z = v[2] - hi.z; lo.w = v[3] - hi.w;
          const uint32_t o = kmaj_off(m, k4, KS);
          *reinterpret_cast<float4*>(A_hi + o) = hi;
          *reinterpret_cast<float4*>(A_lo + o) = lo;
        }
        mbar_arrive(empty_r + 8 * sr);  // this thread's reads of the snapshot stage are done
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(aready + 8 * ja);
      }
    }
    if (!ok && m == 0) atomicOr(a.err, 1);
  } else {
    // ------------------------------------------------------------ epilogue: TMEM lane quadrant warp % 4
    // The new accumulator values overwrite the staged old ones in shared
    // memory, and one TMA tensor store per tile writes them back; the stage
    // is released once that store has read it (one tile later).
    const int q = warp & 3, m = q * 32 + lane, et = tid - 192;
    bool ok = true;
    uint32_t k = 0;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++k) {
      const int sa = k % NSA, jt = k & 1;
      if (ACC == 3) {
        // dot mode: the staged rows are only read, so the stage is released
        // as soon as every thread holds its point's values; the gradient row
        // goes back with one plain store per thread
        if (!mbar_wait_abort(full_a + 8 * sa, (k / NSA) & 1, abort_flag)) { ok = false; break; }
        const float* sP = reinterpret_cast<const float*>(astage0 + sa * C::ASTAGE);
        float ub[GRP];
#pragma unroll
        for (int i = 0; i < GRP; ++i) ub[i] = i < a.r ? sP[i * TILE_M + m] : 0.f;
        const float gold = sP[GRP * TILE_M + m];
        mbar_arrive(empty_a + 8 * sa);
        if (!mbar_wait_abort(mdone + 8 * jt, (k / 2) & 1, abort_flag)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(jt * 32);
        float dot = 0.f;
#pragma unroll
        for (int c = 0; c < GRP / 16; ++c) {
          if (c * 16 < NP) {
            float acc[16];
            tmem_ld16(trow + (uint32_t)(c * 16), acc);
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (c * 16 + j < a.r) dot = fmaf(ub[c * 16 + j], acc[j], dot);
          }
        }
        a.G[shot * a.g_ss + tile_base(tile) + m] = gold + dot;
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mbar_arrive(tfree + 8 * jt);
        continue;
      }
      // each thread waits for itself; the barrier before the store takes the
      // abort decision for all of them at once
      bool w = mbar_wait_abort(full_a + 8 * sa, (k / NSA) & 1, abort_flag);
      if (w) w = mbar_wait_abort(mdone + 8 * jt, (k / 2) & 1, abort_flag);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      float* sP = reinterpret_cast<float*>(astage0 + sa * C::ASTAGE);
      __nv_bfloat16* sPh = reinterpret_cast<__nv_bfloat16*>(sP);
      const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(jt * 32);
#pragma unroll
      for (int c = 0; c < GRP / 16; ++c) {
        if (w && c * 16 < NP) {
          float acc[16];
          tmem_ld16(trow + (uint32_t)(c * 16), acc);
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int i = c * 16 + j;
            if (i < a.r) {
              if (ACC == 0) {
                sP[i * TILE_M + m] += acc[j];
              } else {
                float old = __bfloat162float(sPh[i * TILE_M + m]);
                if (ACC == 2) old += __bfloat162float(sPh[(a.r + i) * TILE_M + m]);  // compensations follow the values
                const float nv = old + acc[j];
                const __nv_bfloat16 hv = __float2bfloat16_rn(nv);
                sPh[i * TILE_M + m] = hv;
                // compensation: the rounding error of the stored value
                if (ACC == 2) sPh[(a.r + i) * TILE_M + m] = __float2bfloat16_rn(nv - __bfloat162float(hv));
              }
            }
          }
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      // the tile's new values are in the stage and its TMEM columns are read
      if (bar_or(2, TILE_M, !w)) { ok = false; break; }
      if (et == 0) {
        mbar_arrive(tfree + 8 * jt);
        const long long row = tile / nxt;
        const int c0 = HX + (int)(tile % nxt) * TILE_M, c1 = (int)(row % a.L.ny) + cy, c2 = (int)(row / a.L.ny) + H;
        tma_store_rows(&mA, c0, c1, c2, shot * (ACC == 2 ? 2 * a.r : a.r), smem_u32(sP));
        bulk_wait_read_all_but_one();  // the previous tile's store has read its stage
        if (k >= 1) mbar_arrive(empty_a + 8 * ((k - 1) % NSA));
      }
    }
    if (et == 0) {
      bulk_wait_all();
      if (!ok) atomicOr(a.err, 1);
    }
  }
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(WS_TMEM_COLS));
  }
}

template <int KP, int ACC>
cudaError_t launch_ws(const GemmArgs& a, cudaStream_t s) {
  using C = WCfg<KP, ACC>;
  static_assert(C::SMEM <= 227 * 1024, "shared memory of the pipelined GEMM");
  const int NP = std::max(16, (a.r + 15) / 16 * 16);
  const cudaError_t e = smem_limit_once<probe_gemm_ws<KP, ACC>>((int)C::SMEM);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long ntiles = (long long)a.L.nz * a.L.ny * ((a.L.nx + TILE_M - 1) / TILE_M);
  // one CTA per SM, the SMs shared among the shots: each persistent CTA then
  // loops over many tiles of its shot (a full SM count per shot made one short
  // wave of CTAs per shot, dominated by pipeline fill and drain)
  const long long grid_x = std::min<long long>(ntiles, std::max<long long>(1, (long long)sms / a.nshots));
  dim3 grid((unsigned)grid_x, a.nshots);
  // the window's sub-tiles of KS levels, each split where the ring wraps
  SubTiles sub{};
  sub.nsub = (a.nlev + KS - 1) / KS;
  const int esize = (ACC == 1 || ACC == 2) ? 2 : 4;
  const int nacc = ACC == 2 ? 2 * a.r : a.r;
  CUtensorMap mR[MAXSUB][2], mA, mG;
  for (int j = 0; j < MAXSUB; ++j) {
    const int jj = j < sub.nsub ? j : 0;  // unused sub-tiles: copies of the first's maps
    sub.rows[j] = std::min(KS, a.nlev - KS * jj);
    sub.slot[j] = (a.level0 + KS * jj) % a.nslots;
    sub.n1[j] = std::min(sub.rows[j], a.nslots - sub.slot[j]);
    const int n2 = sub.rows[j] - sub.n1[j];
    if (!encode_field_map(a.L, a.ring, (long long)a.nshots * a.nslots, 4, TILE_M, 1, sub.n1[j], &mR[j][0]) ||
        !encode_field_map(a.L, a.ring, (long long)a.nshots * a.nslots, 4, TILE_M, 1, n2 > 0 ? n2 : 1, &mR[j][1]))
      return cudaErrorInvalidValue;
  }
  if (!encode_field_map(a.L, a.P, (long long)a.nshots * nacc, esize, TILE_M, 1, nacc, &mA) ||
      !encode_field_map(a.L, ACC == 3 ? (const void*)a.G : a.P, a.nshots, 4, TILE_M, 1, 1, &mG))
    return cudaErrorInvalidValue;
  probe_gemm_ws<KP, ACC><<<grid, WS_THREADS, C::SMEM, s>>>(mR[0][0], mR[0][1], mR[1][0], mR[1][1], mR[2][0],
                                                             mR[2][1], mR[3][0], mR[3][1], mA, mG, a, NP, ntiles,
                                                             sub);
  return cudaGetLastError();
}

template <int KP, int PC>
cudaError_t launch_kp(const GemmArgs& a, cudaStream_t s) {
  const int NP = std::max(16, (a.r + 15) / 16 * 16);
  int ncols = 32;
  while (ncols < NP) ncols <<= 1;
  const size_t smem = (size_t)2 * TILE_M * KP * 4 + (size_t)2 * NP * KP * 4 + 16;
  const cudaError_t e = smem_limit_once<probe_gemm_tf32<KP, PC>>(227 * 1024);
  if (e != cudaSuccess) return e;
  static const int regs = [] {  // the same on every device of this architecture
    cudaFuncAttributes fa;
    return cudaFuncGetAttributes(&fa, probe_gemm_tf32<KP, PC>) == cudaSuccess ? std::max(fa.numRegs, 1) : 255;
  }();
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // CTAs per SM: registers, shared memory (228 KB, 1 KB reserved per CTA), TMEM columns
  const int by_regs = 65536 / (((regs + 7) / 8 * 8) * TILE_M);
  const int by_smem = (int)((228 * 1024) / (smem + 1024));
  const int by_tmem = 512 / ncols;
  const int occ = std::max(1, std::min(std::min(by_regs, by_smem), std::min(by_tmem, 8)));
  const long long ntiles = (long long)a.L.nz * a.L.ny * ((a.L.nx + TILE_M - 1) / TILE_M);
  const long long grid_x = std::min<long long>(ntiles, std::max<long long>(1, (long long)sms * occ / a.nshots));
  dim3 grid((unsigned)grid_x, a.nshots);
  probe_gemm_tf32<KP, PC><<<grid, TILE_M, smem, s>>>(a, NP, ncols, ntiles);
  return cudaGetLastError();
}

}  // namespace

int gemm_kpad(int T) { return T <= 32 ? 32 : (T <= 64 ? 64 : 128); }

cudaError_t launch_probe_gemm(const GemmArgs& a, cudaStream_t s) {
  if (a.nlev <= 0) return cudaSuccess;
  prof_before(2, s);  // TP_KERNEL_PROBE_GEMM
  cudaError_t e;
  if (a.acc != 0 || a.r <= GRP) {  // bf16 storage and dot mode exist on this path only (r <= 32)
#define TP_WS(KPV) (a.acc == 0 ? launch_ws<KPV, 0>(a, s)                                    \
                           : (a.acc == 1 ? launch_ws<KPV, 1>(a, s)                         \
                                         : (a.acc == 2 ? launch_ws<KPV, 2>(a, s) : launch_ws<KPV, 3>(a, s))))
    e = a.nlev <= 32 ? TP_WS(32) : (a.nlev <= 64 ? TP_WS(64) : TP_WS(128));
#undef TP_WS
  } else {  // r > 32 (e.g. identity probes): the register-staged kernel, T <= 64
    e = a.nlev <= 32 ? launch_kp<32, 0>(a, s) : launch_kp<64, 0>(a, s);
  }
  prof_after(2, s);
  return e;
}

}  // namespace tp
