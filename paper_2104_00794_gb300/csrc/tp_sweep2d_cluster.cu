// Persistent 2-D time stepping on thread-block clusters (sm_103a).
//
// Algorithm 1 lines 1 and 5 (operators f and f^T) for a batch of 2-D shots,
// many time steps per launch.  A 2-D shot is small (801 x 301 points: 1 MB
// per level), so one cluster of up to 16 CTAs holds a whole shot's state in
// shared memory and steps it without a round trip through L2 or a kernel
// launch per step:
//   * CTA k of a cluster owns a band of rpc grid rows.  Its shared memory
//     holds the band of the current and the previous level (ping-pong: the
//     new level overwrites the previous one point by point), rows of
//     4 + nx + 4 floats with zero columns for the x stencil;
//   * z neighbours beyond the band are read from the neighbouring CTAs'
//     shared memory (distributed shared memory, generic loads through
//     cluster-mapped addresses), rows outside the grid from a zero row;
//   * one step is: compute the band's new level (results kept in registers
//     until every load of the step is issued), __syncthreads, add the
//     sources of the step (one thread per distinct node, entries at a node
//     summed in index order: deterministic), one cluster barrier;
//   * every level is also copied to its slot of a ring in global memory (the
//     window GEMM of the probe accumulation reads it, and the next launch
//     restarts from it) by asynchronous bulk copies of its rows, issued when
//     the next step starts: the cluster barrier's release would wait for
//     plain global stores, not for these; its receivers are sampled from
//     shared memory;
//   * each thread owns a float4 column of a chunk of the band's rows for the
//     whole launch and marches down it with the z neighbours in a register
//     queue (c2 comes through the read-only cache); rows of the band are read
//     by shared-memory address, rows of other bands through a table of
//     cluster-mapped row addresses;
//   * the cluster size is chosen per grid and device: the least work per CTA
//     over the rounds of clusters the batch needs (at most 16 CTAs).
// Levels form: the arithmetic of the per-step 2-D sweep, operation for
// operation (bit-identical results).  Compensated form (forward only): the
// wavefield is a double-float u + e (e stored as bf16) stepped with an
// error-free transformation, so that the rounding of the stored levels, which
// the Laplacian of the probed field amplifies, is carried instead of lost;
// the Laplacian of u is taken in the per-neighbour difference form, exact for
// neighbours within a factor of two of the centre.
// The kernel has no spin-waits: its only waits are hardware barriers that
// every thread of the cluster reaches the same number of times.
#include <cooperative_groups.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "tp_internal.h"

namespace cg = cooperative_groups;

namespace tp {

namespace {

constexpr int C2_THREADS = 512;
constexpr int C2_MAXCOL = C2_THREADS;  // float4 columns of a band (nx <= 2048)
constexpr int C2_MAXLIST = 1024; // injection or sampling entries of one shot
constexpr int C2_MAXC = 16;      // cluster size limit (non-portable above 8)
constexpr int C2_PER = C2_MAXLIST / C2_THREADS;  // list entries per thread

struct C2Args {
  Layout L;
  Weights W;
  int nshots, C, rpc, sx, nx4;
  int capi, caps;  // capacities of a band's injection and sampling lists (entries)
  int comp, dir, lev0, nsteps, fresh;
  float* ring; int nslots; long long ring_ss;  // level l of shot s: ring + s*ring_ss + (l % nslots)*L.field
  __nv_bfloat16* eslots; long long e_ss;       // comp: e of level l: eslots + s*e_ss + (l % 2)*L.field
  const float* c2;
  const long long* inj_off; const float* inj_coef; int ninj;
  const float* inj_val; long long inj_val_ss; int inj_shift;   // row of the values: new level + inj_shift
  const long long* samp_off; int nsamp;
  float* samp_out; long long samp_out_ss; int samp_shift;      // row of the output: new level + samp_shift
};

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// bf16 <-> fp32 helpers for four values
__device__ __forceinline__ float4 ld_bf4(const __nv_bfloat16* p) {
  const uint2 r = *reinterpret_cast<const uint2*>(p);
  float4 v;
  v.x = __uint_as_float(r.x << 16);
  v.y = __uint_as_float(r.x & 0xffff0000u);
  v.z = __uint_as_float(r.y << 16);
  v.w = __uint_as_float(r.y & 0xffff0000u);
  return v;
}
__device__ __forceinline__ void st_bf4(__nv_bfloat16* p, float4 v) {
  const __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
  uint2 r;
  r.x = *reinterpret_cast<const uint32_t*>(&a);
  r.y = *reinterpret_cast<const uint32_t*>(&b);
  *reinterpret_cast<uint2*>(p) = r;
}

// s = a + b exactly as s + err (Knuth's TwoSum, 6 operations)
__device__ __forceinline__ float two_sum(float a, float b, float* err) {
  const float s = a + b;
  const float bb = s - a;
  *err = (a - (s - bb)) + (b - bb);
  return s;
}

// one row of a band (shared memory) to its place in a global field, as an
// asynchronous bulk copy: the cluster barrier's release does not wait for it
__device__ __forceinline__ void bulk_row_store(float* gdst, const float* ssrc, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst),
               "r"((uint32_t)__cvta_generic_to_shared(ssrc)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the bulk copies of this thread have read their shared memory sources
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// ... and have completed
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// generic-proxy writes to shared memory become visible to the bulk copies
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ float4 lds4(uint32_t a) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
  return v;
}
__device__ __forceinline__ uint2 lds2(uint32_t a) {
  uint2 v;
  asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(a));
  return v;
}
__device__ __forceinline__ float4 bf4(uint2 r) {
  return make_float4(__uint_as_float(r.x << 16), __uint_as_float(r.x & 0xffff0000u), __uint_as_float(r.y << 16),
                     __uint_as_float(r.y & 0xffff0000u));
}

__device__ __forceinline__ float comp4(const float4& v, int p) {
  return p == 0 ? v.x : (p == 1 ? v.y : (p == 2 ? v.z : v.w));
}

template <int R, bool COMP>
__global__ void __launch_bounds__(C2_THREADS, 1) sweep2d_cluster(C2Args a) {
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int ncl = gridDim.x / a.C, cid = blockIdx.x / a.C;
  const int tid = threadIdx.x;
  const int sx = a.sx, sx4 = a.sx / 4, rpc = a.rpc, nx4 = a.nx4;
  const int nz = a.L.nz, nx = a.L.nx, px = a.L.px;
  const int z0 = rank * rpc;
  const int nrow = max(0, min(rpc, nz - z0));  // rows this CTA owns

  // shared memory: both levels of the band, a zero row, the low parts (COMP),
  // row tables, and the band's injection and sampling entries
  extern __shared__ __align__(16) unsigned char smem[];
  float* const U0 = reinterpret_cast<float*>(smem);
  float* const U1 = U0 + (size_t)rpc * sx;
  float* const Z = U1 + (size_t)rpc * sx;  // zeros (as fp32 and as bf16)
  unsigned char* p = reinterpret_cast<unsigned char*>(Z + sx);
  __nv_bfloat16* const E0 = COMP ? reinterpret_cast<__nv_bfloat16*>(p) : nullptr;
  __nv_bfloat16* const E1 = COMP ? E0 + (size_t)rpc * sx : nullptr;
  if (COMP) p = reinterpret_cast<unsigned char*>(E1 + (size_t)rpc * sx);
  const int nrt = rpc + 2 * R;
  const float** rowU = reinterpret_cast<const float**>(p);  // [2][nrt]: rows z0 - R .. z0 + rpc + R - 1
  const __nv_bfloat16** rowE = reinterpret_cast<const __nv_bfloat16**>(rowU + 2 * nrt);
  int* iloc = reinterpret_cast<int*>(rowE + 2 * nrt);  // injection: node (band index)
  int* imeta = iloc + a.capi;                           // k | leader << 16 | (next + 1) << 17
  float* ival = reinterpret_cast<float*>(imeta + a.capi);
  int* sloc = reinterpret_cast<int*>(ival + a.capi);    // sampling: node, column
  int* sk = sloc + a.caps;
  int* cnt = sk + a.caps;  // [0] injection, [1] sampling entries, [4 ..] per-warp counts

  for (int i = tid; i < 2 * nrt; i += C2_THREADS) {
    const int b = i / nrt, zz = z0 - R + i % nrt;
    const float* pu = Z + 4;
    const __nv_bfloat16* pe = reinterpret_cast<const __nv_bfloat16*>(Z) + 4;
    if (zz >= 0 && zz < nz) {
      const int rk = zz / rpc, lr = zz - rk * rpc;
      float* bu = (b ? U1 : U0) + (size_t)lr * sx + 4;
      pu = rk == rank ? bu : cluster.map_shared_rank(bu, rk);
      if (COMP) {
        __nv_bfloat16* be = (b ? E1 : E0) + (size_t)lr * sx + 4;
        pe = rk == rank ? be : cluster.map_shared_rank(be, rk);
      }
    }
    rowU[i] = pu;
    rowE[i] = pe;
  }
  for (int i = tid; i < sx; i += C2_THREADS) Z[i] = 0.f;
  // this thread's points: one float4 column cu of the band, rows [ra, rb);
  // the band's columns are split into nchunk row chunks of hc rows
  const int nchunk = max(1, C2_THREADS / nx4);
  const int hc = (nrow + nchunk - 1) / max(nchunk, 1);
  const int cu = tid % nx4, ch = tid / nx4;
  const int ra = ch < nchunk ? min(nrow, ch * hc) : nrow;
  const int rb = ch < nchunk ? min(nrow, ra + hc) : nrow;
  const uint32_t sU0 = (uint32_t)__cvta_generic_to_shared(U0), sU1 = (uint32_t)__cvta_generic_to_shared(U1);
  const uint32_t sE0 = COMP ? (uint32_t)__cvta_generic_to_shared(E0) : 0u;
  const uint32_t sE1 = COMP ? (uint32_t)__cvta_generic_to_shared(E1) : 0u;

  const float2 m4 = f2(-4.f, -4.f);
  for (int shot = cid; shot < a.nshots; shot += ncl) {
    // ---------------------------------------------------------- per-shot set-up
    // this band's injection and sampling entries, compacted in index order
    for (int list = 0; list < 2; ++list) {
      const int n = list == 0 ? a.ninj : a.nsamp;
      const long long* off = list == 0 ? a.inj_off + (long long)shot * a.ninj
                                       : (n > 0 ? a.samp_off + (long long)shot * a.nsamp : nullptr);
      int* loc = list == 0 ? iloc : sloc;
      int* kk = list == 0 ? imeta : sk;
      if (tid == 0) cnt[list] = 0;
      __syncthreads();
      for (int base = 0; base < n; base += C2_THREADS) {
        const int k = base + tid;
        int l = -1;
        if (k < n) {
          const long long o = off[k];
          if (o >= 0) {
            const int zz = (int)(o / px) - H, xx = (int)(o % px) - HX;
            if (zz >= z0 && zz < z0 + nrow) l = (zz - z0) * sx + 4 + xx;
          }
        }
        const unsigned m = __ballot_sync(0xffffffffu, l >= 0);
        if ((tid & 31) == 0) cnt[4 + (tid >> 5)] = __popc(m);
        __syncthreads();
        int before = 0;
        for (int w = 0; w < (tid >> 5); ++w) before += cnt[4 + w];
        if (l >= 0) {
          const int pos = cnt[list] + before + __popc(m & ((1u << (tid & 31)) - 1u));
          loc[pos] = l;
          kk[pos] = k;
        }
        __syncthreads();
        if (tid == 0) {
          int tot = 0;
          for (int w = 0; w < C2_THREADS / 32; ++w) tot += cnt[4 + w];
          cnt[list] += tot;
        }
        __syncthreads();
      }
    }
    const int ni = cnt[0], ns = cnt[1];
    // coincident injection points: the first entry at a node leads, the
    // others follow it in index order
    float pc[C2_PER];
    int pk[C2_PER];
#pragma unroll
    for (int q = 0; q < C2_PER; ++q) {
      const int i = tid + q * C2_THREADS;
      pc[q] = 0.f;
      pk[q] = 0;
      if (i < ni) {
        int nxt = -1;
        for (int j = i + 1; j < ni; ++j)
          if (iloc[j] == iloc[i]) { nxt = j; break; }
        bool lead = true;
        for (int j = 0; j < i; ++j)
          if (iloc[j] == iloc[i]) { lead = false; break; }
        pk[q] = imeta[i];
        pc[q] = a.inj_coef[(long long)shot * a.ninj + pk[q]];
        imeta[i] = pk[q] | (lead ? 1 << 16 : 0) | ((nxt + 1) << 17);
      }
    }

    // state of the shot: the current and previous levels (and their low parts)
    float* ring = a.ring + (long long)shot * a.ring_ss;
    auto slot = [&](int l) { return (long long)(((l % a.nslots) + a.nslots) % a.nslots) * a.L.field; };
    const int lc0 = a.lev0, lp0 = a.lev0 - a.dir;
    {
      const float* gc = ring + slot(lc0);
      const float* gp = ring + slot(lp0);
      for (int i = tid; i < nrow * sx4; i += C2_THREADS) {
        const int r = i / sx4, c = i % sx4;
        const long long g = (long long)(z0 + r + H) * px + HX - 4 + 4 * c;
        float4 vc = make_float4(0.f, 0.f, 0.f, 0.f), vp = vc;
        if (!a.fresh) {
          vc = *reinterpret_cast<const float4*>(gc + g);
          vp = *reinterpret_cast<const float4*>(gp + g);
        }
        reinterpret_cast<float4*>(U0 + (size_t)r * sx)[c] = vc;
        reinterpret_cast<float4*>(U1 + (size_t)r * sx)[c] = vp;
        if (COMP) {
          float4 ec = make_float4(0.f, 0.f, 0.f, 0.f), ep = ec;
          if (!a.fresh) {
            const __nv_bfloat16* eb = a.eslots + (long long)shot * a.e_ss;
            ec = ld_bf4(eb + (long long)(lc0 & 1) * a.L.field + g);
            ep = ld_bf4(eb + (long long)(lp0 & 1) * a.L.field + g);
          }
          st_bf4(E0 + (size_t)r * sx + 4 * c, ec);
          st_bf4(E1 + (size_t)r * sx + 4 * c, ep);
        }
      }
    }
    // a level (complete since the last cluster barrier) to its ring slot: one
    // bulk copy per row of the band, issued by the first warp
    auto store_level = [&](int lev, const float* Ub) {
      if (tid >= 32) return;
      fence_proxy_async();
      float* g = ring + slot(lev);
      for (int r = tid; r < nrow; r += 32)
        bulk_row_store(g + (long long)(z0 + r + H) * px + HX, Ub + (size_t)r * sx + 4, (uint32_t)(nx4 * 16));
      bulk_commit();
    };
    // receivers of a level (complete since the last cluster barrier)
    auto sample = [&](int lev, const float* Ub) {
      const int orow = lev + a.samp_shift;
      if (orow < 0 || !a.samp_out) return;
      float* out = a.samp_out + (long long)shot * a.samp_out_ss + (long long)orow * a.nsamp;
      for (int i = tid; i < ns; i += C2_THREADS) out[sk[i]] = Ub[sloc[i]];
    };
    cluster.sync();  // every band of the cluster is loaded

    int cur = 0;  // buffer 0 holds the current level, buffer 1 the previous one, then the new one
    for (int step = 0; step < a.nsteps; ++step) {
      const int lcur = a.lev0 + step * a.dir, lnew = lcur + a.dir;
      // values of this step's sources (loaded now, used after the stencil)
      float pv[C2_PER];
#pragma unroll
      for (int q = 0; q < C2_PER; ++q) {
        const int i = tid + q * C2_THREADS;
        pv[q] = i < ni ? pc[q] * __ldg(a.inj_val + (long long)shot * a.inj_val_ss +
                                       (long long)(lnew + a.inj_shift) * a.ninj + pk[q])
                       : 0.f;
      }
      const float* Uc = cur ? U1 : U0;
      float* Un = cur ? U0 : U1;
      __nv_bfloat16* En = cur ? E0 : E1;
      const float** ru = rowU + cur * nrt + R;  // ru[r + d]: row r + d of the current level (any band)
      const __nv_bfloat16** re = rowE + cur * nrt + R;
      // the current level is complete: its receivers, and its copy in the ring
      // (the first level of a launch was stored and sampled by the launch before)
      if (step > 0) {
        store_level(lcur, Uc);
        sample(lcur, Uc);
      }
      // the thread's column chunk, marched down with the z neighbours in a
      // register queue: rows of the band by shared-memory address, rows of
      // other bands (or outside the grid) through the row table
      const uint32_t sUc = cur ? sU1 : sU0, sUn = cur ? sU0 : sU1;
      const uint32_t sEc = cur ? sE1 : sE0, sEn = cur ? sE0 : sE1;
      auto ld_u = [&](int r) -> float4 {
        return (r >= 0 && r < nrow) ? lds4(sUc + (uint32_t)(r * sx + 4 + 4 * cu) * 4u)
                                    : reinterpret_cast<const float4*>(ru[r])[cu];
      };
      auto ld_e = [&](int r) -> float4 {
        return (r >= 0 && r < nrow) ? bf4(lds2(sEc + (uint32_t)(r * sx + 4 + 4 * cu) * 2u))
                                    : bf4(*reinterpret_cast<const uint2*>(re[r] + 4 * cu));
      };
      if (ra < rb) {
        // the queue is circular: row r + d of block row j sits in slot
        // (j + R + d) mod NQ, so whole blocks of NQ rows need no register moves
        constexpr int NQ = 2 * R + 1;
        float4 q[NQ], eq[NQ];
#pragma unroll
        for (int k = 0; k < 2 * R; ++k) {
          q[k] = ld_u(ra - R + k);
          if (COMP) eq[k] = ld_e(ra - R + k);
        }
        const float* c2col = a.c2 + (long long)(z0 + H) * px + HX + 4 * cu;
        for (int r0 = ra; r0 < rb; r0 += NQ) {
#pragma unroll
          for (int j = 0; j < NQ; ++j) {
            const int r = r0 + j;
            if (r < rb) {
              q[(j + 2 * R) % NQ] = ld_u(r + R);
              if (COMP) eq[(j + 2 * R) % NQ] = ld_e(r + R);
              const uint32_t ou = (uint32_t)(r * sx + 4 + 4 * cu);
              const float4 xl = lds4(sUc + (ou - 4) * 4u), xr = lds4(sUc + (ou + 4) * 4u), xc = q[(j + R) % NQ];
              const float4 c1 = lds4(sUn + ou * 4u);  // previous level
              const float4 cq = __ldg(reinterpret_cast<const float4*>(c2col + (long long)r * px));
              const float v[12] = {xl.x, xl.y, xl.z, xl.w, xc.x, xc.y, xc.z, xc.w, xr.x, xr.y, xr.z, xr.w};
              float o[4], en[4] = {0.f, 0.f, 0.f, 0.f};
              if (!COMP) {
                // centred form, the per-step 2-D sweep's operations in its order
                float2 s2[2] = {f2(0.f, 0.f), f2(0.f, 0.f)};
#pragma unroll
                for (int k = 1; k <= R; ++k) {
                  const float4 zp = q[(j + R + k) % NQ], zm = q[(j + R - k) % NQ];
                  const float2 wk = f2(a.W.w[k], a.W.w[k]);
#pragma unroll
                  for (int h = 0; h < 2; ++h) {
                    const int pp = 2 * h;
                    const float2 cv = f2(v[4 + pp], v[5 + pp]);
                    const float2 xs = __fadd2_rn(f2(v[4 + pp + k], v[5 + pp + k]), f2(v[4 + pp - k], v[5 + pp - k]));
                    const float2 zs = __fadd2_rn(h ? f2(zp.z, zp.w) : f2(zp.x, zp.y), h ? f2(zm.z, zm.w) : f2(zm.x, zm.y));
                    s2[h] = __ffma2_rn(wk, __ffma2_rn(m4, cv, __fadd2_rn(xs, zs)), s2[h]);
                  }
                }
                // new = c2 S + (2u - u_prev); 2u is exact, so the FMA rounds 2u - u_prev once, as a subtraction
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                  const int pp = 2 * h;
                  const float2 t = __ffma2_rn(f2(2.f, 2.f), f2(v[4 + pp], v[5 + pp]),
                                              f2(-comp4(c1, pp), -comp4(c1, pp + 1)));
                  const float2 r2 = __ffma2_rn(f2(comp4(cq, pp), comp4(cq, pp + 1)), s2[h], t);
                  o[pp] = r2.x;
                  o[pp + 1] = r2.y;
                }
              } else {
                // double-float levels: U = u + e.  S(u) in the difference form for
                // k = 1, 2 and the centred form for the small weights k = 3, 4; S(e) in
                // the centred form (e is a few ulp of u: its rounding is negligible)
                const float4 el = bf4(lds2(sEc + (ou - 4) * 2u)), er = bf4(lds2(sEc + (ou + 4) * 2u)), ec = eq[(j + R) % NQ];
                const float ve[12] = {el.x, el.y, el.z, el.w, ec.x, ec.y, ec.z, ec.w, er.x, er.y, er.z, er.w};
                const float4 e1 = bf4(lds2(sEn + ou * 2u));
                // two points per packed fp32x2 instruction (each lane the scalar
                // operation of the unpacked form, in the same order)
                float2 su[2] = {f2(0.f, 0.f), f2(0.f, 0.f)}, se[2] = {f2(0.f, 0.f), f2(0.f, 0.f)};
#pragma unroll
                for (int k = 1; k <= R; ++k) {
                  const float4 zp = q[(j + R + k) % NQ], zm = q[(j + R - k) % NQ], ezp = eq[(j + R + k) % NQ],
                               ezm = eq[(j + R - k) % NQ];
                  const float2 wk = f2(a.W.w[k], a.W.w[k]);
#pragma unroll
                  for (int h = 0; h < 2; ++h) {
                    const int pp = 2 * h;
                    const float2 xp = f2(v[4 + pp + k], v[5 + pp + k]), xm = f2(v[4 + pp - k], v[5 + pp - k]);
                    const float2 zpp = h ? f2(zp.z, zp.w) : f2(zp.x, zp.y), zmm = h ? f2(zm.z, zm.w) : f2(zm.x, zm.y);
                    if (k <= 2) {
                      // the two heavy weights: per-neighbour differences, exact
                      // for neighbours within a factor two of the centre
                      const float2 nu = f2(-v[4 + pp], -v[5 + pp]);
                      const float2 dxp = __fadd2_rn(xp, nu), dxm = __fadd2_rn(xm, nu);
                      const float2 dzp = __fadd2_rn(zpp, nu), dzm = __fadd2_rn(zmm, nu);
                      su[h] = __ffma2_rn(wk, __fadd2_rn(__fadd2_rn(dxp, dxm), __fadd2_rn(dzp, dzm)), su[h]);
                    } else {
                      // |w_3|, |w_4| < 0.03: the centred form's rounding is a few
                      // hundredths of an ulp of u here
                      su[h] = __ffma2_rn(wk, __ffma2_rn(m4, f2(v[4 + pp], v[5 + pp]),
                                                        __fadd2_rn(__fadd2_rn(xp, xm), __fadd2_rn(zpp, zmm))),
                                         su[h]);
                    }
                    const float2 xe = __fadd2_rn(f2(ve[4 + pp + k], ve[5 + pp + k]), f2(ve[4 + pp - k], ve[5 + pp - k]));
                    const float2 ze = __fadd2_rn(h ? f2(ezp.z, ezp.w) : f2(ezp.x, ezp.y), h ? f2(ezm.z, ezm.w) : f2(ezm.x, ezm.y));
                    se[h] = __ffma2_rn(wk, __ffma2_rn(m4, f2(ve[4 + pp], ve[5 + pp]), __fadd2_rn(xe, ze)), se[h]);
                  }
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                  const int pp = 2 * h;
                  const float2 two = f2(2.f, 2.f);
                  const float2 uu = f2(v[4 + pp], v[5 + pp]), ee = f2(ve[4 + pp], ve[5 + pp]);
                  const float2 cm = f2(-comp4(c1, pp), -comp4(c1, pp + 1));
                  const float2 em = f2(-comp4(e1, pp), -comp4(e1, pp + 1));
                  const float2 cc2 = f2(comp4(cq, pp), comp4(cq, pp + 1));
                  // 2u - u_prev exactly (TwoSum), then the small terms, then TwoSum again
                  const float2 u2 = __fmul2_rn(two, uu);
                  const float2 av = __fadd2_rn(u2, cm);
                  const float2 bb = __fadd2_rn(av, f2(-u2.x, -u2.y));
                  const float2 ea = __fadd2_rn(__fadd2_rn(u2, f2(-(av.x - bb.x), -(av.y - bb.y))), __fadd2_rn(cm, f2(-bb.x, -bb.y)));
                  const float2 b = __ffma2_rn(cc2, __fadd2_rn(su[h], se[h]), __ffma2_rn(two, ee, em));
                  const float2 bt = __fadd2_rn(b, ea);
                  const float2 sm = __fadd2_rn(av, bt);
                  const float2 b2 = __fadd2_rn(sm, f2(-av.x, -av.y));
                  const float2 er2 = __fadd2_rn(__fadd2_rn(av, f2(-(sm.x - b2.x), -(sm.y - b2.y))), __fadd2_rn(bt, f2(-b2.x, -b2.y)));
                  o[pp] = sm.x;
                  o[pp + 1] = sm.y;
                  en[pp] = er2.x;
                  en[pp + 1] = er2.y;
                }
              }
              if (4 * cu + 3 >= nx) {  // columns past the grid stay zero
#pragma unroll
                for (int pp = 0; pp < 4; ++pp)
                  if (4 * cu + pp >= nx) o[pp] = en[pp] = 0.f;
              }
              // the new value over the previous level (own points: no other thread reads them in this step)
              *reinterpret_cast<float4*>(Un + (size_t)r * sx + 4 + 4 * cu) = make_float4(o[0], o[1], o[2], o[3]);
              if (COMP) st_bf4(En + (size_t)r * sx + 4 + 4 * cu, make_float4(en[0], en[1], en[2], en[3]));
            }
          }
        }
      }
#pragma unroll
      for (int q = 0; q < C2_PER; ++q) {
        const int i = tid + q * C2_THREADS;
        if (i < ni) ival[i] = pv[q];
      }
      if (tid < 32) bulk_wait_read();  // the next step overwrites the buffer the ring copies read
      __syncthreads();
      // sources of this step, into the new level (one thread per node, index order)
      for (int i = tid; i < ni; i += C2_THREADS) {
        const int m = imeta[i];
        if (!(m & (1 << 16))) continue;
        const int l = iloc[i];
        float x = Un[l];
        if (!COMP) {
          for (int j = i; j >= 0; j = (imeta[j] >> 17) - 1) x = x + ival[j];
        } else {
          float e = __bfloat162float(En[l]);
          for (int j = i; j >= 0; j = (imeta[j] >> 17) - 1) {
            float err;
            x = two_sum(x, ival[j], &err);
            e += err;
          }
          En[l] = __float2bfloat16(e);
        }
        Un[l] = x;
      }
      cluster.sync();  // the new level (and its sources) is complete in every band
      cur ^= 1;
    }
    // the last level of the launch: its receivers, its ring slot, and the low
    // parts of the last two levels (the next launch starts from them)
    {
      const int lfin = a.lev0 + a.nsteps * a.dir;
      const float* Uc = cur ? U1 : U0;
      sample(lfin, Uc);
      store_level(lfin, Uc);
      if (COMP) {
        for (int r = ra; r < rb; ++r) {
          const long long go = (long long)(z0 + r + H) * px + HX + 4 * cu;
          __nv_bfloat16* eb = a.eslots + (long long)shot * a.e_ss;
          const __nv_bfloat16* Ef = cur ? E1 : E0;
          const __nv_bfloat16* Ep = cur ? E0 : E1;
          *reinterpret_cast<uint2*>(eb + (long long)(lfin & 1) * a.L.field + go) =
              *reinterpret_cast<const uint2*>(Ef + (size_t)r * sx + 4 + 4 * cu);
          *reinterpret_cast<uint2*>(eb + (long long)((lfin - a.dir) & 1) * a.L.field + go) =
              *reinterpret_cast<const uint2*>(Ep + (size_t)r * sx + 4 + 4 * cu);
        }
      }
    }
    if (tid < 32) bulk_wait_all();  // the ring holds every level of the launch
    cluster.sync();  // no CTA leaves (or starts the next shot) while a neighbour reads its band
  }
}

// list capacity for n entries (a band may hold all of a shot's entries)
int c2_cap(int n) { return (std::max(n, 1) + 3) / 4 * 4; }

size_t c2_smem(int rpc, int sx, int R, bool comp, int capi, int caps) {
  size_t b = (size_t)(2 * rpc + 1) * sx * 4;                // both levels, zero row
  if (comp) b += (size_t)2 * rpc * sx * 2;                  // low parts of both levels (bf16)
  b += (size_t)2 * 2 * (rpc + 2 * R) * sizeof(void*);       // row tables
  b += (size_t)capi * 3 * 4 + (size_t)caps * 2 * 4;         // injection and sampling entries
  b += (size_t)(4 + C2_THREADS / 32) * 4;                   // counts
  return (b + 15) / 16 * 16;
}

// the sizes a band of rpc rows of this grid needs; 0 if it does not fit
size_t c2_fit(const Layout& L, int R, int C, bool comp, int capi, int caps, int* rpc_out) {
  const int nx4 = (L.nx + 3) / 4, sx = 4 * nx4 + 8;
  const int rpc = (L.nz + C - 1) / C;
  if (nx4 > C2_MAXCOL) return 0;
  const size_t sm = c2_smem(rpc, sx, R, comp, capi, caps);
  if (sm > 227 * 1024) return 0;
  *rpc_out = rpc;
  return sm;
}

struct C2Plan {
  int C = 0, rpc = 0, sx = 0, nx4 = 0, ncl = 0;
  size_t smem = 0;
};

// clusters of C CTAs with `smem` bytes each that fit on the current device at once (cached)
template <int R, bool COMP>
int c2_max_clusters(int C, size_t smem) {
  static std::mutex m;
  static std::vector<std::pair<long long, int>> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  const long long key = ((long long)dev << 40) | ((long long)C << 32) | (long long)smem;
  {
    std::lock_guard<std::mutex> lk(m);
    for (auto& e : cache)
      if (e.first == key) return e.second;
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)C);
  cfg.blockDim = dim3(C2_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, sweep2d_cluster<R, COMP>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    n = 0;
  }
  std::lock_guard<std::mutex> lk(m);
  cache.emplace_back(key, n);
  return n;
}

// Cluster size: over the sizes whose bands fit (shared memory, register
// cache), the one with the least work per CTA over the rounds that the
// batch's clusters need on this device (a CTA below 128 items counts as 128).
// The step time follows the work per CTA well below a thread's worth of items:
// a 101 x 101 shot (config 1) ran 3.25 ms per gradient with 3-CTA clusters
// (884 items a CTA), 2.43 ms with 6 (442), 2.10 ms with 12 and 2.05 ms with 16
// (182 items).
template <int R, bool COMP>
C2Plan c2_plan(const Layout& L, int nshots, int capi, int caps) {
  C2Plan best;
  long long best_est = -1;
  for (int C = 1; C <= C2_MAXC; ++C) {
    int rpc = 0;
    const size_t sm = c2_fit(L, R, C, COMP, capi, caps, &rpc);
    if (!sm) continue;
    const int ncl = c2_max_clusters<R, COMP>(C, sm);
    if (ncl < 1) continue;
    const long long rounds = (nshots + ncl - 1) / ncl;
    const long long est = rounds * std::max<long long>((long long)rpc * ((L.nx + 3) / 4), 128);
    if (best_est < 0 || est < best_est) {
      best_est = est;
      best.C = C;
      best.rpc = rpc;
      best.smem = sm;
      best.ncl = ncl;
    }
  }
  best.nx4 = (L.nx + 3) / 4;
  best.sx = 4 * best.nx4 + 8;
  return best;
}

template <int R, bool COMP>
cudaError_t c2_launch(const C2Args& a0, cudaStream_t s) {
  auto kern = sweep2d_cluster<R, COMP>;
  cudaError_t e = smem_limit_once<sweep2d_cluster<R, COMP>>(227 * 1024, true);
  if (e != cudaSuccess) return e;
  const int capi = c2_cap(a0.ninj), caps = c2_cap(a0.nsamp);
  const C2Plan pl = c2_plan<R, COMP>(a0.L, a0.nshots, capi, caps);
  if (!pl.C) return cudaErrorInvalidConfiguration;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)pl.C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)(pl.C * std::min(pl.ncl, a0.nshots)));
  cfg.blockDim = dim3(C2_THREADS);
  cfg.dynamicSmemBytes = pl.smem;
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  C2Args a = a0;
  a.C = pl.C;
  a.rpc = pl.rpc;
  a.sx = pl.sx;
  a.nx4 = pl.nx4;
  a.capi = capi;
  a.caps = caps;
  e = cudaLaunchKernelEx(&cfg, kern, a);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace

bool cluster2d_fits(const Layout& L, const Weights& W, int nshots, int nsrc, int nrec, bool comp) {
  (void)nshots;
  if (L.ndim != 2 || W.sw > 0) return false;
  if (nsrc > C2_MAXLIST || nrec > C2_MAXLIST) return false;
  // the larger of the two sets in both lists covers the forward and the adjoint launches
  const int cap = c2_cap(std::max(nsrc, nrec));
  int rpc = 0;
  for (int C = 1; C <= C2_MAXC; ++C)
    if (c2_fit(L, W.R, C, comp, cap, cap, &rpc)) return true;
  return false;
}

cudaError_t launch_cluster2d(const Cluster2dArgs& c, cudaStream_t s) {
  C2Args a{};
  a.L = c.L;
  a.W = c.W;
  a.nshots = c.nshots;
  a.comp = c.comp;
  a.dir = c.dir;
  a.lev0 = c.lev0;
  a.nsteps = c.nsteps;
  a.fresh = c.fresh;
  a.ring = c.ring; a.nslots = c.nslots; a.ring_ss = c.ring_ss;
  a.eslots = reinterpret_cast<__nv_bfloat16*>(c.eslots); a.e_ss = c.e_ss;
  a.c2 = c.c2;
  a.inj_off = c.inj_off; a.inj_coef = c.inj_coef; a.ninj = c.ninj;
  a.inj_val = c.inj_val; a.inj_val_ss = c.inj_val_ss; a.inj_shift = c.inj_shift;
  a.samp_off = c.samp_off; a.nsamp = c.nsamp;
  a.samp_out = c.samp_out; a.samp_out_ss = c.samp_out_ss; a.samp_shift = c.samp_shift;
  prof_before(0, s);  // TP_KERNEL_STENCIL
  cudaError_t e;
  if (c.W.R == 4) e = c.comp ? c2_launch<4, true>(a, s) : c2_launch<4, false>(a, s);
  else e = c.comp ? c2_launch<2, true>(a, s) : c2_launch<2, false>(a, s);
  prof_after(0, s);
  return e;
}

}  // namespace tp
