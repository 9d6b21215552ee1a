// C ABI of libtprobe (include/tprobe.h): argument checks, workspace layout
// and the host-side time loops that enqueue the kernels.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "tp_internal.h"
#include "tprobe.h"

namespace tp {

namespace {

thread_local std::string g_err;

tp_status fail(tp_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

#define TRY(expr)                                                                           \
  do {                                                                                      \
    cudaError_t e_ = (expr);                                                                \
    if (e_ != cudaSuccess) return fail(TP_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
  } while (0)

long long round_up(long long a, long long b) { return (a + b - 1) / b * b; }

constexpr int NBLK = 1024;       // partial sums of the fp64 reductions
constexpr size_t SCAL_BYTES = 256;  // err flag, vmax bits, fallback scalars

struct Scal {
  int err;
  unsigned int vmax_bits;
  int pad[2];
  double misfit, gnorm;
};

// ------------------------------------------------------------------ profiling
struct Prof {
  std::mutex m;
  bool on = false;
  std::vector<cudaEvent_t> ev;
  std::vector<int> kind;
  size_t used = 0;
  bool open = false;
};
Prof g_prof;

}  // namespace

// Under stream capture a plain event record only marks a dependency; the
// external flag makes it a real record node of the graph, timed at replay.
static void prof_record(cudaEvent_t e, cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cs);
  if (cs == cudaStreamCaptureStatusActive) cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
  else cudaEventRecord(e, s);
}

void prof_before(int kind, cudaStream_t s) {
  if (!g_prof.on) return;
  std::lock_guard<std::mutex> lk(g_prof.m);
  if (!g_prof.on || g_prof.used + 2 > g_prof.ev.size()) return;
  prof_record(g_prof.ev[g_prof.used], s);
  g_prof.kind[g_prof.used / 2] = kind;
  g_prof.open = true;
}

void prof_after(int, cudaStream_t s) {
  if (!g_prof.on) return;
  std::lock_guard<std::mutex> lk(g_prof.m);
  if (!g_prof.on || !g_prof.open) return;
  prof_record(g_prof.ev[g_prof.used + 1], s);
  g_prof.used += 2;
  g_prof.open = false;
}

void set_last_error(const char* msg) { g_err = msg; }

namespace {
std::atomic<long long> g_wait_limit{0};  // 0: the default
}  // namespace

long long wait_limit_cycles() {
  const long long v = g_wait_limit.load(std::memory_order_relaxed);
  return v > 0 ? v : DEFAULT_WAIT_CYCLES;
}

Layout make_layout(int ndim, int nx, int ny, int nz) {
  Layout L;
  L.ndim = ndim;
  L.nx = nx;
  L.ny = ny;
  L.nz = nz;
  // the right x halo of a row is the left padding of the next row (zeros)
  L.px = (int)(HX + round_up(nx, XALIGN));
  L.py = ndim == 3 ? (int)round_up(ny, YALIGN) + 2 * H : 1;
  L.pz = nz + 2 * H;
  L.plane = (long long)L.py * L.px;
  L.field = round_up((long long)L.pz * L.plane + 64, 64);  // + slack: the last row's right halo
  return L;
}

// Centred second-derivative weights (Fornberg 1988, Table 1).
Weights stencil_weights(int order) {
  Weights W{};
  if (order == 4) {
    W.R = 2;
    W.w[0] = -5.0f / 2.0f;
    W.w[1] = 4.0f / 3.0f;
    W.w[2] = -1.0f / 12.0f;
  } else {
    W.R = 4;
    W.w[0] = (float)(-205.0 / 72.0);
    W.w[1] = (float)(8.0 / 5.0);
    W.w[2] = (float)(-1.0 / 5.0);
    W.w[3] = (float)(8.0 / 315.0);
    W.w[4] = (float)(-1.0 / 560.0);
  }
  return W;
}

namespace {

struct Plan {
  int op = 0;
  Layout L{};
  Weights W{};
  int nshots = 0, nsrc = 0, nrec = 0, nt = 0, r = 0, T = 0, S = 0, kind = 0, acc = 0, form = 0;
  bool c2d = false;  // 2-D batch on the persistent cluster path (tp_sweep2d_cluster.cu)
  int comp = 0;      // compensated (double-float) forward
  size_t o_e = 0;    // comp: bf16 low parts of two levels per shot
  float scale = 1.f;
  size_t bytes = 0;
  size_t o_scal = 0, o_part = 0, o_c2 = 0, o_f = 0, o_P = 0, o_V = 0, o_Q = 0, o_d = 0, o_soff = 0, o_roff = 0,
         o_cs = 0, o_cr = 0, o_qbar = 0, o_gacc = 0, o_sacc = 0, o_conv = 0, o_w = 0;
  // deterministic injection groups of the sources and of the receivers
  size_t o_salone = 0, o_ralone = 0, o_sshared = 0, o_rshared = 0, o_sn = 0, o_rn = 0;
  long long nf = 0;  // fields in the wavefield block
  // probed state (Q, then the forward accumulators): offsets inside the state
  // buffer, which tp_gradient_probed places at o_state of its workspace
  size_t s_Q = 0, s_P = 0, state_bytes = 0, o_state = 0;
  long long acc_elems = 0;  // accumulator storage elements per shot (r fields, 2r with compensation)
  size_t acc_esize = 4;     // bytes per stored element
};

size_t take(size_t& cur, size_t bytes) {
  const size_t o = cur;
  cur += (size_t)round_up((long long)bytes, 256);
  return o;
}

tp_status check_grid(const tp_grid* g) {
  if (!g) return fail(TP_ERR_ARG, "grid is NULL");
  if (g->ndim != 2 && g->ndim != 3) return fail(TP_ERR_ARG, "ndim must be 2 or 3 (got %d)", g->ndim);
  if (g->nx < 1 || g->ny < 1 || g->nz < 1) return fail(TP_ERR_ARG, "grid extents must be >= 1");
  if (g->ndim == 2 && g->ny != 1) return fail(TP_ERR_ARG, "2-D grids need ny == 1 (got %d)", g->ny);
  if (g->order != 4 && g->order != 8) return fail(TP_ERR_ARG, "order must be 4 or 8 (got %d)", g->order);
  if (!(g->h > 0.f) || !(g->dt > 0.f)) return fail(TP_ERR_ARG, "h and dt must be positive");
  if (g->nt < 3) return fail(TP_ERR_ARG, "nt must be >= 3 (got %d)", g->nt);
  if ((long long)g->nx * g->ny * g->nz > (1LL << 40)) return fail(TP_ERR_ARG, "grid too large");
  if (g->nx > (1 << 24) || g->nz > (1 << 24) || g->ny > (1 << 24)) return fail(TP_ERR_ARG, "grid extent too large");
  if (!(g->vmax >= 0.f)) return fail(TP_ERR_ARG, "vmax must be >= 0");
  if (g->form != TP_FORM_LEVELS && g->form != TP_FORM_INCREMENT && g->form != TP_FORM_COMPENSATED)
    return fail(TP_ERR_ARG, "unknown time form %d", g->form);
  if (g->sponge < 0 || !(g->sponge_eta >= 0.f) || !std::isfinite(g->sponge_eta))
    return fail(TP_ERR_ARG, "sponge width must be >= 0 and sponge_eta finite and >= 0");
  return TP_OK;
}

tp_status check_geom(const tp_geom* g) {
  if (!g) return fail(TP_ERR_ARG, "geom is NULL");
  if (g->nshots < 1 || g->nsrc < 1 || g->nrec < 1) return fail(TP_ERR_ARG, "nshots, nsrc, nrec must be >= 1");
  if (!g->src || !g->rec) return fail(TP_ERR_ARG, "src/rec index arrays are NULL");
  if ((long long)g->nshots * g->nrec > (1LL << 31) || (long long)g->nshots * g->nsrc > (1LL << 31))
    return fail(TP_ERR_ARG, "too many sources or receivers");
  return TP_OK;
}

tp_status check_probe(const tp_probe* p, int nt) {
  if (!p) return fail(TP_ERR_ARG, "probe is NULL");
  if (p->acc < TP_ACC_F32 || p->acc > TP_ACC_F32_FOLD) return fail(TP_ERR_ARG, "unknown accumulator type %d", p->acc);
  if (p->acc != TP_ACC_F32 && p->r > 32)
    return fail(TP_ERR_ARG, "bf16 and folded accumulators need r <= 32 (got %d)", p->r);
  if (p->kind < 0 || p->kind > 3) return fail(TP_ERR_ARG, "unknown probe kind %d", p->kind);
  if (p->r < 1 || p->r > 256) return fail(TP_ERR_ARG, "r must be in 1..256 (got %d)", p->r);
  if (p->kind == TP_PROBE_IDENTITY && p->r != nt) return fail(TP_ERR_ARG, "identity probes need r == nt");
  if (p->kind == TP_PROBE_USER && !p->Z_user) return fail(TP_ERR_ARG, "user probes need Z_user");
  if (p->T != 32 && p->T != 64 && p->T != 128) return fail(TP_ERR_ARG, "window T must be 32, 64 or 128 (got %d)", p->T);
  if (p->T == 128 && p->r > 32) return fail(TP_ERR_ARG, "window T = 128 needs r <= 32 (got %d)", p->r);
  if (!(p->scale >= 0.f)) return fail(TP_ERR_ARG, "scale must be >= 0");
  return TP_OK;
}

tp_status make_plan(int op, const tp_grid* g, const tp_geom* geo, const tp_probe* pr, Plan* P) {
  tp_status st = check_grid(g);
  if (st != TP_OK) return st;
  if ((st = check_geom(geo)) != TP_OK) return st;
  if (op < TP_OP_FORWARD || op > TP_OP_PROBED_BACKWARD) return fail(TP_ERR_ARG, "unknown op %d", op);
  const bool probed = op == TP_OP_GRADIENT_PROBED || op == TP_OP_PROBED_FORWARD || op == TP_OP_PROBED_BACKWARD;
  if (probed && (st = check_probe(pr, g->nt)) != TP_OK) return st;
  P->op = op;
  P->L = make_layout(g->ndim, g->nx, g->ny, g->nz);
  P->W = stencil_weights(g->order);
  P->W.sw = g->sponge_eta > 0.f ? g->sponge : 0;
  P->W.samax = (float)(0.5 * (double)g->sponge_eta * (double)g->dt);
  P->nshots = geo->nshots;
  P->nsrc = geo->nsrc;
  P->nrec = geo->nrec;
  P->nt = g->nt;
  const size_t fb = (size_t)P->L.field * sizeof(float);
  const long long ns = P->nshots;
  size_t cur = 0;
  P->o_scal = take(cur, SCAL_BYTES);
  P->o_part = take(cur, NBLK * sizeof(double));
  P->o_soff = take(cur, (size_t)ns * P->nsrc * sizeof(long long));
  P->o_roff = take(cur, (size_t)ns * P->nrec * sizeof(long long));
  P->o_cs = take(cur, (size_t)ns * P->nsrc * sizeof(float));
  P->o_cr = take(cur, (size_t)ns * P->nrec * sizeof(float));
  P->o_salone = take(cur, (size_t)ns * P->nsrc);
  P->o_ralone = take(cur, (size_t)ns * P->nrec);
  P->o_sshared = take(cur, (size_t)ns * P->nsrc * sizeof(int));
  P->o_rshared = take(cur, (size_t)ns * P->nrec * sizeof(int));
  P->o_sn = take(cur, (size_t)ns * sizeof(int));
  P->o_rn = take(cur, (size_t)ns * sizeof(int));
  P->o_c2 = take(cur, fb);
  P->form = g->form;
  P->comp = g->form == TP_FORM_COMPENSATED;
  P->c2d = g->form != TP_FORM_INCREMENT && cluster2d_fits(P->L, P->W, P->nshots, P->nsrc, P->nrec, P->comp);
  if (P->comp && !P->c2d)
    return fail(TP_ERR_ARG, "the compensated form needs a 2-D grid without an absorbing layer whose shot fits one "
                            "thread-block cluster, with at most 1024 sources and receivers per shot");
  if (P->comp) P->o_e = take(cur, (size_t)2 * ns * P->L.field * 2);  // bf16 low parts, two levels per shot
  if (P->form == TP_FORM_INCREMENT) P->o_w = take(cur, (size_t)ns * fb);  // the increment field of each shot
  switch (op) {
    case TP_OP_FORWARD:
    case TP_OP_ADJOINT:
      P->nf = 3 * ns;
      P->o_f = take(cur, (size_t)P->nf * fb);
      break;
    case TP_OP_GRADIENT_PROBED:
    case TP_OP_PROBED_FORWARD:
    case TP_OP_PROBED_BACKWARD: {
      P->kind = pr->kind;
      P->r = pr->r;
      P->T = pr->T;
      P->S = P->T + 2;
      P->acc = pr->acc;
      P->scale = pr->scale > 0.f ? pr->scale
                                 : ((pr->kind == TP_PROBE_RADEMACHER || pr->kind == TP_PROBE_GAUSSIAN) ? 1.0f / pr->r : 1.0f);
      P->acc_esize = (P->acc == TP_ACC_F32 || P->acc == TP_ACC_F32_FOLD) ? 4 : 2;
      P->acc_elems = (long long)P->r * P->L.field * (P->acc == TP_ACC_BF16_KAHAN ? 2 : 1);
      const size_t accb = (size_t)ns * P->acc_elems * P->acc_esize;  // one accumulator set, all shots
      size_t sc = 0;
      P->s_Q = take(sc, (size_t)ns * P->nt * P->r * sizeof(float));
      P->s_P = take(sc, accb);
      P->state_bytes = sc;
      P->nf = (long long)P->S * ns;
      P->o_f = take(cur, (size_t)P->nf * fb);  // ring of T+2 levels
      if (op != TP_OP_PROBED_FORWARD) {
        if (P->acc != TP_ACC_F32_FOLD) P->o_V = take(cur, accb);  // vbar (the folded form keeps none)
        P->o_qbar = take(cur, (size_t)ns * P->nsrc * P->r * sizeof(float));
        P->o_gacc = take(cur, (size_t)ns * fb);
        if (P->acc == TP_ACC_BF16 || P->acc == TP_ACC_BF16_KAHAN)
          P->o_conv = take(cur, (size_t)2 * ns * fb);  // fp32 copies of P_i, V_i
      }
      if (op == TP_OP_GRADIENT_PROBED) {
        P->o_state = take(cur, P->state_bytes);
        P->o_d = take(cur, (size_t)ns * P->nt * P->nrec * sizeof(float));
      }
      break;
    }
    case TP_OP_GRADIENT_FULL:
      P->nf = (long long)P->nt * ns;
      P->o_f = take(cur, (size_t)P->nf * fb);   // forward history, levels 0..nt-1
      P->o_P = take(cur, (size_t)3 * ns * fb);  // adjoint levels
      P->o_d = take(cur, (size_t)ns * P->nt * P->nrec * sizeof(float));
      P->o_gacc = take(cur, (size_t)ns * fb);
      P->o_sacc = take(cur, (size_t)ns * P->nsrc * sizeof(double));
      break;
  }
  P->bytes = cur;
  return TP_OK;
}

// Courant number above which the leapfrog scheme with this Laplacian grows:
// (v dt / h)^2 * ndim * |S(pi)| <= 4, S(pi) the 1-D stencil symbol at Nyquist.
double cfl_limit(const Plan& P) {
  double sym = P.W.w[0];
  for (int k = 1; k <= P.W.R; ++k) sym += 2.0 * P.W.w[k] * ((k & 1) ? -1.0 : 1.0);
  return 2.0 / std::sqrt(P.L.ndim * std::fabs(sym));
}

// A family of padded fields in the workspace: `nfields` consecutive fields at
// byte offset `off`, shot s's copy of field f at index f + s * fs.
struct Fam {
  size_t off;
  int nfields;
  int fs;
};

struct Ctx {
  const Plan& P;
  char* ws;
  cudaStream_t st;
  template <class T> T* at(size_t o) const { return reinterpret_cast<T*>(ws + o); }
  Scal* scal() const { return at<Scal>(P.o_scal); }
  int* err() const { return &scal()->err; }
  float* field(size_t base, long long i) const { return at<float>(base) + i * P.L.field; }
  float* ptr(const Fam& f, int f0) const { return field(f.off, f0); }
  long long ss(const Fam& f) const { return (long long)f.fs * P.L.field; }
  FieldRef ref(const Fam& f, int f0) const { return FieldRef{at<float>(f.off), f.nfields, f0, f.fs}; }
};

tp_status check_ws(const Plan& P, void* ws, size_t ws_bytes) {
  if (!ws) return fail(TP_ERR_ARG, "workspace is NULL");
  if (reinterpret_cast<uintptr_t>(ws) % 256) return fail(TP_ERR_ARG, "workspace must be 256-byte aligned");
  if (ws_bytes < P.bytes) return fail(TP_ERR_NOMEM, "workspace of %zu bytes, %zu needed", ws_bytes, P.bytes);
  return TP_OK;
}

// Common set-up: coefficient field, point offsets, CFL check.
tp_status setup(const Ctx& c, const tp_grid* g, const tp_geom* geo, const float* vel) {
  const Plan& P = c.P;
  if (!vel) return fail(TP_ERR_ARG, "vel is NULL");
  TRY(cudaMemsetAsync(c.scal(), 0, SCAL_BYTES, c.st));
  TRY(cudaMemsetAsync(c.at<float>(P.o_c2), 0, (size_t)P.L.field * sizeof(float), c.st));
  const double dt2 = (double)g->dt * (double)g->dt;
  TRY(launch_prep_c2(P.L, vel, dt2 / ((double)g->h * (double)g->h), c.at<float>(P.o_c2), c.st));
  TRY(launch_prep_points(P.L, P.W, geo->src, (long long)P.nshots * P.nsrc, vel, dt2, c.at<long long>(P.o_soff),
                         c.at<float>(P.o_cs), c.err(), c.st));
  TRY(launch_prep_points(P.L, P.W, geo->rec, (long long)P.nshots * P.nrec, vel, dt2, c.at<long long>(P.o_roff),
                         c.at<float>(P.o_cr), c.err(), c.st));
  // injection groups; the wavefield block (at least one field per shot, zeroed
  // by every operation after the set-up) serves as the count scratch
  int* cnt = c.at<int>(P.o_f);
  TRY(launch_point_groups(c.at<long long>(P.o_soff), P.nsrc, P.nshots, P.L.field, cnt, c.at<unsigned char>(P.o_salone),
                          c.at<int>(P.o_sshared), c.at<int>(P.o_sn), c.st));
  TRY(launch_point_groups(c.at<long long>(P.o_roff), P.nrec, P.nshots, P.L.field, cnt, c.at<unsigned char>(P.o_ralone),
                          c.at<int>(P.o_rshared), c.at<int>(P.o_rn), c.st));
  float vmax = g->vmax;
  if (!(vmax > 0.f)) {
    TRY(launch_vmax(vel, (long long)g->nx * g->ny * g->nz, &c.scal()->vmax_bits, c.st));
    Scal host{};
    TRY(cudaMemcpyAsync(&host, c.scal(), sizeof(Scal), cudaMemcpyDeviceToHost, c.st));
    TRY(cudaStreamSynchronize(c.st));
    if (host.err & 2) return fail(TP_ERR_ARG, "a source or receiver index lies outside the grid");
    uint32_t bits = host.vmax_bits;
    memcpy(&vmax, &bits, sizeof(vmax));
  }
  const double courant = (double)vmax * g->dt / g->h;
  if (!(courant <= cfl_limit(P)))
    return fail(TP_ERR_UNSTABLE, "CFL: vmax*dt/h = %.4f exceeds the stability limit %.4f", courant, cfl_limit(P));
  return TP_OK;
}

// the increment fields (TP_FORM_INCREMENT), one per shot
Fam inc_fam(const Plan& P) { return Fam{P.o_w, P.nshots, 1}; }

tp_status step(const Ctx& c, const Fam& f, int cur, int old, int out) {
  const FieldRef c2 = c.ref(Fam{c.P.o_c2, 1, 0}, 0);
  if (c.P.form == TP_FORM_INCREMENT) {
    const Fam fw = inc_fam(c.P);
    StencilArgs a{c.ref(f, cur), c.ref(fw, 0), c2, c.ptr(f, out), c.ss(f), c.P.nshots, c.ptr(fw, 0), c.ss(fw)};
    TRY(launch_stencil(MODE_INC, c.P.L, c.P.W, a, c.st, c.err()));
  } else {
    StencilArgs a{c.ref(f, cur), c.ref(f, old), c2, c.ptr(f, out), c.ss(f), c.P.nshots};
    TRY(launch_stencil(MODE_STEP, c.P.L, c.P.W, a, c.st, c.err()));
  }
  return TP_OK;
}

// sampling of `samp` at offsets soff into out (may be null), injection into `inj`
tp_status point(const Ctx& c, const float* samp, long long samp_ss, const long long* soff, int nsamp, float* out,
                long long out_ss, float* inj, long long inj_ss, const long long* ioff, const float* icoef, int ninj,
                const float* ival, long long ival_ss, double* acc = nullptr, const float* aval = nullptr,
                long long aval_ss = 0) {
  PointArgs a{};
  a.nshots = c.P.nshots;
  a.field_samp = samp; a.samp_ss = samp_ss; a.samp_off = soff; a.nsamp = samp ? nsamp : 0;
  a.samp_out = out; a.samp_out_ss = out_ss;
  a.field_inj = inj; a.inj_ss = inj_ss; a.inj_off = ioff; a.inj_coef = icoef; a.ninj = inj ? ninj : 0;
  if (inj) {  // the groups of the set whose offsets ioff are
    const bool src = ioff == c.at<long long>(c.P.o_soff);
    a.inj_alone = c.at<unsigned char>(src ? c.P.o_salone : c.P.o_ralone);
    a.inj_shared = c.at<int>(src ? c.P.o_sshared : c.P.o_rshared);
    a.inj_nshared = c.at<int>(src ? c.P.o_sn : c.P.o_rn);
  }
  if (inj && c.P.form == TP_FORM_INCREMENT) {  // sources enter the increment as well as the new level
    a.field_inj2 = c.ptr(inc_fam(c.P), 0);
    a.inj2_ss = c.ss(inc_fam(c.P));
  }
  a.inj_val = ival; a.inj_val_ss = ival_ss;
  a.acc = acc; a.acc_val = aval; a.acc_val_ss = aval_ss;
  TRY(launch_point(a, c.st));
  return TP_OK;
}

#define TRYS(expr)                    \
  do {                                \
    tp_status s_ = (expr);            \
    if (s_ != TP_OK) return s_;       \
  } while (0)

// Arguments of a persistent 2-D launch over family f (level l of a shot in
// slot l mod f.fs: every family passed to the loops below stores level t at
// level(t) = t mod f.fs).
Cluster2dArgs cluster_args(const Ctx& c, const Fam& f, int dir, int lev0, int nsteps, bool fresh, int comp) {
  const Plan& P = c.P;
  Cluster2dArgs a{};
  a.L = P.L;
  a.W = P.W;
  a.nshots = P.nshots;
  a.comp = comp;
  a.dir = dir;
  a.lev0 = lev0;
  a.nsteps = nsteps;
  a.fresh = fresh ? 1 : 0;
  a.ring = c.at<float>(f.off);
  a.nslots = f.fs;
  a.ring_ss = c.ss(f);
  a.eslots = comp ? c.at<char>(P.o_e) : nullptr;
  a.e_ss = 2 * P.L.field;
  a.c2 = c.at<float>(P.o_c2);
  return a;
}

// Forward loop (Algorithm 1 lines 0-3).  Level t of every shot lives in
// field level(t) of family f.  d (may be null) receives R u[t];
// after_level(t) runs once level t is complete (sources injected).  On the
// 2-D cluster path the steps between two levels that closes() marks (the
// levels after which after_level launches work) run as one persistent launch
// that samples and injects by itself.
template <class LevelFn, class AfterFn, class ClosesFn>
tp_status forward_loop(const Ctx& c, const Fam& f, LevelFn level, const float* wav, float* d, AfterFn after_level,
                       ClosesFn closes) {
  const Plan& P = c.P;
  const long long dss = (long long)P.nt * P.nrec, wss = (long long)P.nt * P.nsrc, ss = c.ss(f);
  if (P.c2d) {
    if (P.comp) TRY(cudaMemsetAsync(c.at<char>(P.o_e), 0, (size_t)2 * P.nshots * P.L.field * 2, c.st));
    for (int t = 1; t <= P.nt - 2;) {
      int te = t;
      while (te < P.nt - 2 && !closes(te + 1)) ++te;
      Cluster2dArgs a = cluster_args(c, f, +1, t, te - t + 1, t == 1, P.comp);
      a.inj_off = c.at<long long>(P.o_soff); a.inj_coef = c.at<float>(P.o_cs); a.ninj = P.nsrc;
      a.inj_val = wav; a.inj_val_ss = wss; a.inj_shift = -1;  // q[t] enters level t + 1
      if (d) {
        a.samp_off = c.at<long long>(P.o_roff); a.nsamp = P.nrec;
        a.samp_out = d; a.samp_out_ss = dss; a.samp_shift = 0;
      }
      TRY(launch_cluster2d(a, c.st));
      for (int lev = t + 1; lev <= te + 1; ++lev) TRYS(after_level(lev));
      t = te + 1;
    }
    return TP_OK;
  }
  if (P.form == TP_FORM_INCREMENT)  // u[1] - u[0] = 0
    TRY(cudaMemsetAsync(c.at<char>(P.o_w), 0, (size_t)P.nshots * P.L.field * sizeof(float), c.st));
  for (int t = 1; t <= P.nt - 2; ++t) {
    TRYS(step(c, f, level(t), level(t - 1), level(t + 1)));
    TRYS(point(c, d ? c.ptr(f, level(t)) : nullptr, ss, c.at<long long>(P.o_roff), P.nrec,
               d ? d + (long long)t * P.nrec : nullptr, dss, c.ptr(f, level(t + 1)), ss, c.at<long long>(P.o_soff),
               c.at<float>(P.o_cs), P.nsrc, wav + (long long)t * P.nsrc, wss));
    TRYS(after_level(t + 1));
  }
  if (d)
    TRYS(point(c, c.ptr(f, level(P.nt - 1)), ss, c.at<long long>(P.o_roff), P.nrec, d + (long long)(P.nt - 1) * P.nrec,
               dss, nullptr, 0, nullptr, nullptr, 0, nullptr, 0));
  return TP_OK;
}

// Adjoint loop (Algorithm 1 lines 4-7) driven by s[nshots][nt][nrec].
// q_out (may be null) receives S lambda[t+1] at row t; acc/aval accumulate
// sum_k lambda[k][src] q[k-1] for the full gradient's source term.  Without
// acc, a 2-D batch runs on the cluster path as in forward_loop (levels form).
// step_j (optional) replaces the plain step that forms level j.
template <class LevelFn, class AfterFn, class ClosesFn, class StepFn = std::nullptr_t>
tp_status adjoint_loop(const Ctx& c, const Fam& f, LevelFn level, const float* s, float* q_out, double* acc,
                       const float* aval, AfterFn after_level, ClosesFn closes, StepFn step_j = nullptr) {
  const Plan& P = c.P;
  const long long sss = (long long)P.nt * P.nrec, qss = (long long)P.nt * P.nsrc, ss = c.ss(f);
  const bool samp = q_out || acc;
  if (P.c2d && !acc) {
    for (int j = P.nt - 1; j >= 2;) {
      int je = j;
      while (je > 2 && !closes(je)) --je;
      Cluster2dArgs a = cluster_args(c, f, -1, j + 1, j - je + 1, j == P.nt - 1, 0);
      a.inj_off = c.at<long long>(P.o_roff); a.inj_coef = c.at<float>(P.o_cr); a.ninj = P.nrec;
      a.inj_val = s; a.inj_val_ss = sss; a.inj_shift = 0;  // s[j] enters lambda[j]
      if (q_out) {
        a.samp_off = c.at<long long>(P.o_soff); a.nsamp = P.nsrc;
        a.samp_out = q_out; a.samp_out_ss = qss; a.samp_shift = -1;  // (F^T s)[j - 1] = S lambda[j]
      }
      TRY(launch_cluster2d(a, c.st));
      for (int lev = j; lev >= je; --lev) TRYS(after_level(lev));
      j = je - 1;
    }
    return TP_OK;
  }
  if (P.form == TP_FORM_INCREMENT)  // lambda[nt] - lambda[nt+1] = 0
    TRY(cudaMemsetAsync(c.at<char>(P.o_w), 0, (size_t)P.nshots * P.L.field * sizeof(float), c.st));
  for (int j = P.nt - 1; j >= 2; --j) {
    if constexpr (std::is_same_v<StepFn, std::nullptr_t>)
      TRYS(step(c, f, level(j + 1), level(j + 2), level(j)));
    else
      TRYS(step_j(j));
    TRYS(point(c, samp ? c.ptr(f, level(j + 1)) : nullptr, ss, c.at<long long>(P.o_soff), P.nsrc,
               q_out ? q_out + (long long)j * P.nsrc : nullptr, qss, c.ptr(f, level(j)), ss, c.at<long long>(P.o_roff),
               c.at<float>(P.o_cr), P.nrec, s + (long long)j * P.nrec, sss, acc,
               aval ? aval + (long long)j * P.nsrc : nullptr, qss));
    TRYS(after_level(j));
  }
  if (samp)
    TRYS(point(c, c.ptr(f, level(2)), ss, c.at<long long>(P.o_soff), P.nsrc, q_out ? q_out + P.nsrc : nullptr, qss,
               nullptr, 0, nullptr, nullptr, 0, nullptr, 0, acc, aval ? aval + P.nsrc : nullptr, qss));
  return TP_OK;
}

tp_status misfit_and_residual(const Ctx& c, float* d, const float* dobs, double* misfit) {
  const Plan& P = c.P;
  if (!dobs) return fail(TP_ERR_ARG, "d_obs is NULL");
  double* part = c.at<double>(P.o_part);
  TRY(launch_residual(d, dobs, (long long)P.nshots * P.nt * P.nrec, part, NBLK, c.st));
  TRY(launch_finalize_sum(part, NBLK, 0.5, misfit ? misfit : &c.scal()->misfit, 0, c.err(), c.st));
  return TP_OK;
}

tp_status grad_norm(const Ctx& c, const float* grad, double* gnorm) {
  const Plan& P = c.P;
  double* part = c.at<double>(P.o_part);
  TRY(launch_sumsq(grad, (long long)P.L.nx * P.L.ny * P.L.nz, part, NBLK, c.st));
  TRY(launch_finalize_sum(part, NBLK, 1.0, gnorm ? gnorm : &c.scal()->gnorm, 1, c.err(), c.st));
  return TP_OK;
}

}  // namespace
}  // namespace tp

using namespace tp;

extern "C" {

tp_status tp_form_supported(const tp_grid* grid, const tp_geom* geom) {
  TRYS(check_grid(grid));
  if (!geom) return fail(TP_ERR_ARG, "geom is NULL");
  if (geom->nshots < 1 || geom->nsrc < 1 || geom->nrec < 1) return fail(TP_ERR_ARG, "nshots, nsrc, nrec must be >= 1");
  if (grid->form == TP_FORM_COMPENSATED) {
    const Layout L = make_layout(grid->ndim, grid->nx, grid->ny, grid->nz);
    Weights W = stencil_weights(grid->order);
    W.sw = grid->sponge_eta > 0.f ? grid->sponge : 0;
    if (!cluster2d_fits(L, W, geom->nshots, geom->nsrc, geom->nrec, true))
      return fail(TP_ERR_ARG, "the compensated form needs a 2-D grid without an absorbing layer whose shot fits one "
                              "thread-block cluster, with at most 1024 sources and receivers per shot");
  }
  return TP_OK;
}

size_t tp_workspace_bytes(int op, const tp_grid* grid, const tp_geom* geom, const tp_probe* probe) {
  Plan P;
  if (make_plan(op, grid, geom, probe, &P) != TP_OK) return 0;
  return P.bytes;
}

tp_status tp_forward(const tp_grid* grid, const tp_geom* geom, const float* vel, const float* wavelet, float* d_out,
                     void* ws, size_t ws_bytes, void* stream) {
  Plan P;
  TRYS(make_plan(TP_OP_FORWARD, grid, geom, nullptr, &P));
  TRYS(check_ws(P, ws, ws_bytes));
  if (!wavelet || !d_out) return fail(TP_ERR_ARG, "wavelet/d_out is NULL");
  Ctx c{P, static_cast<char*>(ws), static_cast<cudaStream_t>(stream)};
  TRYS(setup(c, grid, geom, vel));
  TRY(cudaMemsetAsync(c.at<float>(P.o_f), 0, (size_t)P.nf * P.L.field * sizeof(float), c.st));
  TRY(cudaMemsetAsync(d_out, 0, (size_t)P.nshots * P.nt * P.nrec * sizeof(float), c.st));
  const Fam f{P.o_f, (int)P.nf, 3};
  auto level = [](int t) { return t % 3; };
  TRYS(forward_loop(c, f, level, wavelet, d_out, [](int) { return TP_OK; }, [](int) { return false; }));
  return TP_OK;
}

tp_status tp_adjoint(const tp_grid* grid, const tp_geom* geom, const float* vel, const float* d_in, float* q_out,
                     void* ws, size_t ws_bytes, void* stream) {
  Plan P;
  TRYS(make_plan(TP_OP_ADJOINT, grid, geom, nullptr, &P));
  TRYS(check_ws(P, ws, ws_bytes));
  if (!d_in || !q_out) return fail(TP_ERR_ARG, "d_in/q_out is NULL");
  Ctx c{P, static_cast<char*>(ws), static_cast<cudaStream_t>(stream)};
  TRYS(setup(c, grid, geom, vel));
  TRY(cudaMemsetAsync(c.at<float>(P.o_f), 0, (size_t)P.nf * P.L.field * sizeof(float), c.st));
  TRY(cudaMemsetAsync(q_out, 0, (size_t)P.nshots * P.nt * P.nsrc * sizeof(float), c.st));
  const Fam f{P.o_f, (int)P.nf, 3};
  auto level = [](int t) { return t % 3; };
  TRYS(adjoint_loop(c, f, level, d_in, q_out, nullptr, nullptr, [](int) { return TP_OK; }, [](int) { return false; }));
  return TP_OK;
}

}  // extern "C"

namespace tp {
namespace {

// adjoint windows: levels top .. bottom with top = nt - 1 - k T, bottom =
// max(2, top - T + 1); a window closes at its bottom level
auto adj_window_closes(int nt, int T) {
  return [=](int lev) {
    const int top = nt - 1 - ((nt - 1 - lev) / T) * T;
    return lev == std::max(2, top - T + 1);
  };
}

GemmArgs gemm_args(const Ctx& c, float* Q) {
  const Plan& P = c.P;
  GemmArgs g{};
  g.ring = c.at<float>(P.o_f); g.slot_stride = P.L.field; g.ring_ss = (long long)P.S * P.L.field; g.nslots = P.S;
  g.Q = Q; g.nt = P.nt; g.r = P.r; g.q_ss = (long long)P.nt * P.r;
  g.L = P.L; g.pstride = P.L.field; g.p_ss = P.acc_elems;
  g.acc = P.acc == TP_ACC_F32_FOLD ? TP_ACC_F32 : P.acc;  // the folded form accumulates ubar in fp32
  g.nshots = P.nshots; g.qlo = 2; g.qhi = P.nt - 1;
  g.q_has_lo = (P.kind == TP_PROBE_GAUSSIAN || P.kind == TP_PROBE_USER) ? 1 : 0;
  g.err = c.err();
  return g;
}

// Algorithm 1 lines 0-3: forward sweep; d (all shots, zeroed here) receives
// R u[t]; the accumulators Pacc receive P_i = sum_{j=2}^{nt-2} Q[j+1, i] u[j]
// (windows of T levels), from which ubar_i = v^2 (L P_i + S^T qbar_i).
tp_status probed_forward_impl(const Ctx& c, const tp_probe* probe, const float* wavelet, float* d, float* Q,
                              void* Pacc) {
  const Plan& P = c.P;
  const size_t fb = (size_t)P.L.field * sizeof(float);
  const int nt = P.nt, T = P.T, S = P.S;
  TRY(cudaMemsetAsync(c.at<float>(P.o_f), 0, (size_t)P.nf * fb, c.st));
  TRY(cudaMemsetAsync(Pacc, 0, (size_t)P.nshots * P.acc_elems * P.acc_esize, c.st));
  TRY(cudaMemsetAsync(d, 0, (size_t)P.nshots * nt * P.nrec * sizeof(float), c.st));
  TRY(launch_probes(P.kind, nt, P.r, probe->seed, 0, P.nshots, probe->Z_user, Q, c.st));
  const Fam ring{P.o_f, (int)P.nf, S};
  auto level = [S](int t) { return t % S; };
  GemmArgs g = gemm_args(c, Q);
  g.P = Pacc;
  g.qshift = 1;
  const int jlast = nt - 2;
  // a window of levels w0 .. w0 + T - 1 (from level 2; the last one ends at nt - 2) closes at its last level
  auto closes = [=](int lev) {
    if (lev < 2 || lev > jlast) return false;
    const int w0 = 2 + ((lev - 2) / T) * T;
    return lev == std::min(w0 + T - 1, jlast);
  };
  auto fwd_after = [&](int lev) -> tp_status {
    if (closes(lev)) {
      const int w0 = 2 + ((lev - 2) / T) * T;
      g.level0 = w0;
      g.nlev = lev - w0 + 1;
      TRY(launch_probe_gemm(g, c.st));
    }
    return TP_OK;
  };
  return forward_loop(c, ring, level, wavelet, d, fwd_after, closes);
}

// Single-accumulator form (TP_ACC_F32_FOLD): ubar_i = c2 S(P_i) + dt^2 v^2 S^T qbar_i
// (= dt^2 v^2 (L P_i + S^T qbar_i)) replaces P_i in place; the adjoint windows
// fold sum_i ubar_i (Q_w^T lambda)_i into one accumulator field per shot, and
// grad = -(scale / dt^2) sum_s of it.  Same estimator as the two-set form.
tp_status probed_backward_fold(const Ctx& c, const tp_grid* grid, const tp_geom* geom, const float* vel,
                               const float* wavelet, const float* s, int wrt_velocity, float* grad, double* gnorm,
                               const float* Q, float* Pacc) {
  const Plan& P = c.P;
  const size_t fb = (size_t)P.L.field * sizeof(float);
  const int nt = P.nt, T = P.T, S = P.S, r = P.r;
  const Fam fG{P.o_gacc, P.nshots, 1};
  float* tmp = c.ptr(fG, 0);  // scratch for ubar_i until the adjoint needs the accumulator
  TRY(launch_qbar(Q, nt, r, wavelet, P.nsrc, P.nshots, 1, nt - 2, 1, c.at<float>(P.o_qbar), c.st));
  const FieldRef fPr{Pacc, (int)(P.nshots * (long long)r), 0, r};
  const FieldRef c2 = c.ref(Fam{P.o_c2, 1, 0}, 0);
  for (int i = 0; i < r; ++i) {
    FieldRef pi = fPr;
    pi.f0 = i;
    TRY(cudaMemsetAsync(tmp, 0, (size_t)P.nshots * fb, c.st));
    StencilArgs a{pi, c2, c.ref(fG, 0), tmp, c.ss(fG), P.nshots};
    TRY(launch_stencil(MODE_IMAGE, P.L, P.W, a, c.st, c.err()));
    TRY(cudaMemcpy2DAsync(Pacc + (long long)i * P.L.field, (size_t)P.acc_elems * sizeof(float), tmp, fb, fb,
                          P.nshots, cudaMemcpyDeviceToDevice, c.st));
  }
  TRY(launch_source_into_acc(c.at<long long>(P.o_soff), geom->src, vel, (double)grid->dt * (double)grid->dt,
                             c.at<float>(P.o_qbar), P.nsrc, P.nshots, r, Pacc, P.acc_elems, P.L.field, c.st));
  TRY(cudaMemsetAsync(c.at<float>(P.o_f), 0, (size_t)P.nf * fb, c.st));  // levels nt, nt+1 start at zero
  TRY(cudaMemsetAsync(tmp, 0, (size_t)P.nshots * fb, c.st));
  const Fam ring{P.o_f, (int)P.nf, S};
  auto level = [S](int t) { return t % S; };
  GemmArgs g = gemm_args(c, const_cast<float*>(Q));
  g.P = Pacc;
  g.acc = 3;  // dot epilogue
  g.G = tmp;
  g.g_ss = P.L.field;
  g.qshift = 0;
  auto adj_after = [&](int lev) -> tp_status {
    const int top = nt - 1 - ((nt - 1 - lev) / T) * T;
    const int bottom = std::max(2, top - T + 1);
    if (lev == bottom) {
      g.level0 = bottom;
      g.nlev = top - bottom + 1;
      TRY(launch_probe_gemm(g, c.st));
    }
    return TP_OK;
  };
  TRYS(adjoint_loop(c, ring, level, s, nullptr, nullptr, nullptr, adj_after, adj_window_closes(nt, T)));
  TRY(launch_finish_grad(P.L, vel, tmp, P.nshots, P.L.field, P.scale / (grid->dt * grid->dt), grad, c.st, 0));
  if (wrt_velocity) TRY(launch_chain_velocity(vel, grad, (long long)P.L.nx * P.L.ny * P.L.nz, c.st));
  TRYS(grad_norm(c, grad, gnorm));
  return TP_OK;
}

// Algorithm 1 lines 4-7 with the two-set accumulators: the adjoint sweep
// driven by s (all shots) and vbar_i = sum_{k=2}^{nt-1} Q[k, i] lambda[k]
// into the workspace's V block.
tp_status adjoint_probes(const Ctx& c, const float* s, const float* Q) {
  const Plan& P = c.P;
  const size_t fb = (size_t)P.L.field * sizeof(float);
  const int nt = P.nt, T = P.T, S = P.S;
  TRY(cudaMemsetAsync(c.at<float>(P.o_f), 0, (size_t)P.nf * fb, c.st));  // levels nt, nt+1 start at zero
  TRY(cudaMemsetAsync(c.at<char>(P.o_V), 0, (size_t)P.nshots * P.acc_elems * P.acc_esize, c.st));
  const Fam ring{P.o_f, (int)P.nf, S};
  auto level = [S](int t) { return t % S; };
  GemmArgs g = gemm_args(c, const_cast<float*>(Q));
  g.P = c.at<char>(P.o_V);
  g.qshift = 0;
  auto adj_after = [&](int lev) -> tp_status {
    const int top = nt - 1 - ((nt - 1 - lev) / T) * T;
    const int bottom = std::max(2, top - T + 1);
    if (lev == bottom) {
      g.level0 = bottom;
      g.nlev = top - bottom + 1;
      TRY(launch_probe_gemm(g, c.st));
    }
    return TP_OK;
  };
  return adjoint_loop(c, ring, level, s, nullptr, nullptr, nullptr, adj_after, adj_window_closes(nt, T));
}

// Algorithm 1 lines 4-8: adjoint sweep driven by s (all shots), vbar_i =
// sum_{k=2}^{nt-1} Q[k, i] lambda[k], then grad = -scale sum_i ubar_i vbar_i
// (dJ/dm, or dJ/dv when wrt_velocity) and its fp64 norm.
tp_status probed_backward_impl(const Ctx& c, const tp_grid* grid, const tp_geom* geom, const float* vel,
                               const float* wavelet, const float* s, int wrt_velocity, float* grad, double* gnorm,
                               const float* Q, const void* Pacc) {
  const Plan& P = c.P;
  if (P.acc == TP_ACC_F32_FOLD)
    return probed_backward_fold(c, grid, geom, vel, wavelet, s, wrt_velocity, grad, gnorm, Q,
                                static_cast<float*>(const_cast<void*>(Pacc)));
  const size_t fb = (size_t)P.L.field * sizeof(float);
  const int nt = P.nt, r = P.r;
  TRY(cudaMemsetAsync(c.at<float>(P.o_gacc), 0, (size_t)P.nshots * fb, c.st));
  TRYS(adjoint_probes(c, s, Q));

  // combine (Algorithm 1 line 8): ubar = v^2 (L P + S^T qbar), grad = -scale sum_i ubar vbar
  const Fam fG{P.o_gacc, P.nshots, 1};
  if (P.acc == TP_ACC_F32) {
    const size_t vo = P.o_V;
    const long long accf = P.nshots * (long long)r;
    // the state's accumulators and the workspace's vbar as field families
    const FieldRef fPr{static_cast<const float*>(Pacc), (int)accf, 0, r};
    const Fam fV{vo, (int)accf, r};
    for (int i = 0; i < r; ++i) {
      FieldRef pi = fPr;
      pi.f0 = i;
      StencilArgs a{pi, c.ref(fV, i), c.ref(fG, 0), c.ptr(fG, 0), c.ss(fG), P.nshots};
      TRY(launch_stencil(MODE_IMAGE, P.L, P.W, a, c.st, c.err()));
    }
  } else {
    // bf16 storage: fp32 copies of P_i and V_i (per shot) feed the same sweep
    const Fam fC{P.o_conv, 2 * P.nshots, 1};
    float* cP = c.ptr(fC, 0);
    float* cV = c.ptr(fC, P.nshots);
    for (int i = 0; i < r; ++i) {
      TRY(launch_acc_to_f32(Pacc, P.acc, r, i, P.L.field, P.nshots, cP, P.L.field, c.st));
      TRY(launch_acc_to_f32(c.at<char>(P.o_V), P.acc, r, i, P.L.field, P.nshots, cV, P.L.field, c.st));
      StencilArgs a{c.ref(fC, 0), c.ref(fC, P.nshots), c.ref(fG, 0), c.ptr(fG, 0), c.ss(fG), P.nshots};
      TRY(launch_stencil(MODE_IMAGE, P.L, P.W, a, c.st, c.err()));
    }
  }
  TRY(launch_finish_grad(P.L, vel, c.at<float>(P.o_gacc), P.nshots, P.L.field, P.scale / (grid->h * grid->h), grad,
                         c.st));
  TRY(launch_qbar(Q, nt, r, wavelet, P.nsrc, P.nshots, 1, nt - 2, 1, c.at<float>(P.o_qbar), c.st));
  TRY(launch_source_term(P.L, vel, geom->src, c.at<long long>(P.o_soff), P.nsrc, P.nshots, P.scale,
                         c.at<float>(P.o_qbar), c.at<char>(P.o_V), P.acc, r, P.acc_elems, nullptr, grad, c.st));
  if (wrt_velocity) TRY(launch_chain_velocity(vel, grad, (long long)P.L.nx * P.L.ny * P.L.nz, c.st));
  TRYS(grad_norm(c, grad, gnorm));
  return TP_OK;
}

tp_status check_state(const Plan& P, void* state, size_t state_bytes) {
  if (!state) return fail(TP_ERR_ARG, "state is NULL");
  if (reinterpret_cast<uintptr_t>(state) % 256) return fail(TP_ERR_ARG, "state must be 256-byte aligned");
  if (state_bytes < P.state_bytes)
    return fail(TP_ERR_NOMEM, "state of %zu bytes, %zu needed", state_bytes, P.state_bytes);
  return TP_OK;
}

}  // namespace
}  // namespace tp

extern "C" {

tp_status tp_gradient_probed(const tp_grid* grid, const tp_geom* geom, const tp_probe* probe, const float* vel,
                             const float* wavelet, const float* d_obs, float* grad, double* misfit, double* gnorm,
                             void* ws, size_t ws_bytes, void* stream) {
  Plan P;
  TRYS(make_plan(TP_OP_GRADIENT_PROBED, grid, geom, probe, &P));
  TRYS(check_ws(P, ws, ws_bytes));
  if (!wavelet || !d_obs || !grad) return fail(TP_ERR_ARG, "wavelet/d_obs/grad is NULL");
  Ctx c{P, static_cast<char*>(ws), static_cast<cudaStream_t>(stream)};
  TRYS(setup(c, grid, geom, vel));
  char* state = c.at<char>(P.o_state);
  float* Q = reinterpret_cast<float*>(state + P.s_Q);
  void* Pacc = state + P.s_P;
  float* d = c.at<float>(P.o_d);
  TRYS(probed_forward_impl(c, probe, wavelet, d, Q, Pacc));
  TRYS(misfit_and_residual(c, d, d_obs, misfit));
  TRYS(probed_backward_impl(c, grid, geom, vel, wavelet, d, 0, grad, gnorm, Q, Pacc));
  return TP_OK;
}

size_t tp_probed_state_bytes(const tp_grid* grid, const tp_geom* geom, const tp_probe* probe) {
  Plan P;
  if (make_plan(TP_OP_PROBED_FORWARD, grid, geom, probe, &P) != TP_OK) return 0;
  return P.state_bytes;
}

tp_status tp_probed_forward(const tp_grid* grid, const tp_geom* geom, const tp_probe* probe, const float* vel,
                            const float* wavelet, float* d_out, void* state, size_t state_bytes, void* ws,
                            size_t ws_bytes, void* stream) {
  Plan P;
  TRYS(make_plan(TP_OP_PROBED_FORWARD, grid, geom, probe, &P));
  TRYS(check_ws(P, ws, ws_bytes));
  TRYS(check_state(P, state, state_bytes));
  if (!wavelet || !d_out) return fail(TP_ERR_ARG, "wavelet/d_out is NULL");
  Ctx c{P, static_cast<char*>(ws), static_cast<cudaStream_t>(stream)};
  TRYS(setup(c, grid, geom, vel));
  char* st = static_cast<char*>(state);
  return probed_forward_impl(c, probe, wavelet, d_out, reinterpret_cast<float*>(st + P.s_Q), st + P.s_P);
}

tp_status tp_probed_backward(const tp_grid* grid, const tp_geom* geom, const tp_probe* probe, const float* vel,
                             const float* wavelet, const float* adj_src, int wrt_velocity, float* grad, double* gnorm,
                             void* state, size_t state_bytes, void* ws, size_t ws_bytes, void* stream) {
  Plan P;
  TRYS(make_plan(TP_OP_PROBED_BACKWARD, grid, geom, probe, &P));
  TRYS(check_ws(P, ws, ws_bytes));
  TRYS(check_state(P, state, state_bytes));
  if (!wavelet || !adj_src || !grad) return fail(TP_ERR_ARG, "wavelet/adj_src/grad is NULL");
  Ctx c{P, static_cast<char*>(ws), static_cast<cudaStream_t>(stream)};
  TRYS(setup(c, grid, geom, vel));
  const char* st = static_cast<const char*>(state);
  return probed_backward_impl(c, grid, geom, vel, wavelet, adj_src, wrt_velocity, grad, gnorm,
                              reinterpret_cast<const float*>(st + P.s_Q), st + P.s_P);
}

size_t tp_residual_workspace_bytes(void) { return NBLK * sizeof(double) + SCAL_BYTES; }

tp_status tp_residual(float* d, const float* d_obs, int64_t n, double* misfit, void* ws, size_t ws_bytes,
                      void* stream) {
  if (!d || !d_obs || !misfit) return fail(TP_ERR_ARG, "d/d_obs/misfit is NULL");
  if (n < 1) return fail(TP_ERR_ARG, "n must be >= 1");
  if (!ws) return fail(TP_ERR_ARG, "workspace is NULL");
  if (reinterpret_cast<uintptr_t>(ws) % 256) return fail(TP_ERR_ARG, "workspace must be 256-byte aligned");
  if (ws_bytes < tp_residual_workspace_bytes())
    return fail(TP_ERR_NOMEM, "workspace of %zu bytes, %zu needed", ws_bytes, tp_residual_workspace_bytes());
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* part = static_cast<double*>(ws);
  Scal* sc = reinterpret_cast<Scal*>(static_cast<char*>(ws) + NBLK * sizeof(double));
  TRY(cudaMemsetAsync(sc, 0, SCAL_BYTES, st));
  // the reduction of the fused gradient call (misfit_and_residual), on the caller's buffers
  TRY(launch_residual(d, d_obs, (long long)n, part, NBLK, st));
  TRY(launch_finalize_sum(part, NBLK, 0.5, misfit, 0, &sc->err, st));
  return TP_OK;
}

tp_status tp_probed_image(const tp_grid* grid, const tp_geom* geom, const tp_probe* probe, const float* vel,
                          const float* adj_src, int cond, float* image, const void* state, size_t state_bytes,
                          void* ws, size_t ws_bytes, void* stream) {
  Plan P;
  TRYS(make_plan(TP_OP_PROBED_BACKWARD, grid, geom, probe, &P));
  TRYS(check_ws(P, ws, ws_bytes));
  TRYS(check_state(P, const_cast<void*>(state), state_bytes));
  if (!adj_src || !image) return fail(TP_ERR_ARG, "adj_src/image is NULL");
  if (cond != TP_IMAGE_CORRELATION && cond != TP_IMAGE_GRADIENT) return fail(TP_ERR_ARG, "unknown imaging condition %d", cond);
  if (P.acc != TP_ACC_F32) return fail(TP_ERR_ARG, "imaging conditions need TP_ACC_F32 accumulators");
  Ctx c{P, static_cast<char*>(ws), static_cast<cudaStream_t>(stream)};
  TRYS(setup(c, grid, geom, vel));
  const char* st = static_cast<const char*>(state);
  TRYS(adjoint_probes(c, adj_src, reinterpret_cast<const float*>(st + P.s_Q)));
  TRY(launch_image(P.L, grid->order, grid->h, cond, reinterpret_cast<const float*>(st + P.s_P), P.acc_elems,
                   c.at<float>(P.o_V), P.acc_elems, P.r, P.nshots, P.scale, image, c.st));
  return TP_OK;
}

tp_status tp_gradient_full(const tp_grid* grid, const tp_geom* geom, const float* vel, const float* wavelet,
                           const float* d_obs, float* grad, double* misfit, double* gnorm, void* ws, size_t ws_bytes,
                           void* stream) {
  Plan P;
  TRYS(make_plan(TP_OP_GRADIENT_FULL, grid, geom, nullptr, &P));
  TRYS(check_ws(P, ws, ws_bytes));
  if (!wavelet || !d_obs || !grad) return fail(TP_ERR_ARG, "wavelet/d_obs/grad is NULL");
  Ctx c{P, static_cast<char*>(ws), static_cast<cudaStream_t>(stream)};
  TRYS(setup(c, grid, geom, vel));
  const size_t fb = (size_t)P.L.field * sizeof(float);
  const int nt = P.nt;
  TRY(cudaMemsetAsync(c.at<float>(P.o_f), 0, (size_t)P.nf * fb, c.st));
  TRY(cudaMemsetAsync(c.at<float>(P.o_P), 0, (size_t)3 * P.nshots * fb, c.st));
  TRY(cudaMemsetAsync(c.at<float>(P.o_gacc), 0, (size_t)P.nshots * fb, c.st));
  TRY(cudaMemsetAsync(c.at<double>(P.o_sacc), 0, (size_t)P.nshots * P.nsrc * sizeof(double), c.st));
  float* d = c.at<float>(P.o_d);
  TRY(cudaMemsetAsync(d, 0, (size_t)P.nshots * nt * P.nrec * sizeof(float), c.st));
  const Fam fh{P.o_f, (int)P.nf, nt}, fl{P.o_P, 3 * P.nshots, 3}, fG{P.o_gacc, P.nshots, 1};
  auto hist = [](int t) { return t; };
  TRYS(forward_loop(c, fh, hist, wavelet, d, [](int) { return TP_OK; }, [](int) { return false; }));
  TRYS(misfit_and_residual(c, d, d_obs, misfit));
  // adjoint with the imaging condition of Eq. 3 in its stencil form:
  // gacc_s += lambda_s[j] * S(u_s[j-1])   (udd[j] = v^2 (L u[j-1] + S^T q[j-1]))
  auto lam = [](int k) { return k % 3; };
  if (P.L.ndim == 3 && P.form == TP_FORM_LEVELS) {
    // 3-D: in the sweep of the step that forms lambda[j], whose source field
    // lambda[j+1] is complete: the terms j+1 = nt .. 3 in the same order and
    // the same arithmetic as the separate sweep (lambda[nt] = 0 and u[1] = 0
    // make the first and the omitted last term exactly zero)
    const FieldRef c2 = c.ref(Fam{P.o_c2, 1, 0}, 0);
    auto fused = [&](int j) -> tp_status {
      StencilArgs a{c.ref(fl, lam(j + 1)), c.ref(fl, lam(j + 2)), c2, c.ptr(fl, lam(j)), c.ss(fl), P.nshots};
      a.img = c.ref(fh, j);
      a.gin = c.ref(fG, 0);
      a.gout = c.ptr(fG, 0);
      a.gout_ss = c.ss(fG);
      TRY(launch_stencil(MODE_STEP_IMG, P.L, P.W, a, c.st, c.err()));
      return TP_OK;
    };
    TRYS(adjoint_loop(c, fl, lam, d, nullptr, c.at<double>(P.o_sacc), wavelet, [](int) { return TP_OK; },
                      [](int) { return true; }, fused));
  } else {
    auto imaging = [&](int j) -> tp_status {
      StencilArgs a{c.ref(fh, j - 1), c.ref(fl, lam(j)), c.ref(fG, 0), c.ptr(fG, 0), c.ss(fG), P.nshots};
      TRY(launch_stencil(MODE_IMAGE, P.L, P.W, a, c.st, c.err()));
      return TP_OK;
    };
    TRYS(adjoint_loop(c, fl, lam, d, nullptr, c.at<double>(P.o_sacc), wavelet, imaging, [](int) { return true; }));
  }
  TRY(launch_finish_grad(P.L, vel, c.at<float>(P.o_gacc), P.nshots, P.L.field, 1.0f / (grid->h * grid->h), grad,
                         c.st));
  TRY(launch_source_term(P.L, vel, geom->src, c.at<long long>(P.o_soff), P.nsrc, P.nshots, 1.0f, nullptr, nullptr, 0,
                         0, 0, c.at<double>(P.o_sacc), grad, c.st));
  TRYS(grad_norm(c, grad, gnorm));
  return TP_OK;
}

tp_status tp_probes(const tp_probe* probe, int nt, int shot, float* Z, void* stream) {
  if (nt < 1) return fail(TP_ERR_ARG, "nt must be >= 1");
  TRYS(check_probe(probe, nt));
  if (!Z || shot < 0) return fail(TP_ERR_ARG, "Z is NULL or shot < 0");
  const float* zu = probe->Z_user ? probe->Z_user + (long long)shot * nt * probe->r : nullptr;
  TRY(launch_probes(probe->kind, nt, probe->r, probe->seed, shot, 1, zu, Z, static_cast<cudaStream_t>(stream)));
  return TP_OK;
}

tp_status tp_workspace_status(void* ws, size_t ws_bytes, void* stream) {
  if (!ws || ws_bytes < SCAL_BYTES) return fail(TP_ERR_ARG, "workspace is NULL or too small");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int flag = 0;
  TRY(cudaMemcpyAsync(&flag, ws, sizeof(int), cudaMemcpyDeviceToHost, st));
  TRY(cudaStreamSynchronize(st));
  TRY(cudaMemsetAsync(ws, 0, sizeof(int), st));
  if (flag & 1) return fail(TP_ERR_TIMEOUT, "a bounded device-side wait timed out");
  if (flag & 2) return fail(TP_ERR_ARG, "a source or receiver index lies outside the grid");
  if (flag & 4) return fail(TP_ERR_ARG, "the record is numerically rank deficient for r range-finding probes");
  return TP_OK;
}

const char* tp_last_error(void) { return g_err.c_str(); }

tp_status tp_set_wait_limit(int64_t cycles) {
  if (cycles < 0) return fail(TP_ERR_ARG, "the wait limit must be >= 0 (got %lld)", (long long)cycles);
  g_wait_limit.store(cycles, std::memory_order_relaxed);
  return TP_OK;
}

tp_status tp_profile_begin(int max_launches) {
  std::lock_guard<std::mutex> lk(g_prof.m);
  if (g_prof.on) return fail(TP_ERR_ARG, "profiling already active");
  const size_t n = (size_t)(max_launches > 0 ? max_launches : 65536);
  if (g_prof.ev.size() < 2 * n) {
    size_t have = g_prof.ev.size();
    g_prof.ev.resize(2 * n);
    for (size_t i = have; i < 2 * n; ++i) TRY(cudaEventCreate(&g_prof.ev[i]));
  }
  g_prof.kind.assign(n, 0);
  g_prof.used = 0;
  g_prof.open = false;
  g_prof.on = true;
  return TP_OK;
}

tp_status tp_profile_end(double* ms, int64_t* launches) {
  std::lock_guard<std::mutex> lk(g_prof.m);
  if (!g_prof.on) return fail(TP_ERR_ARG, "profiling not active");
  g_prof.on = false;
  for (int k = 0; k < TP_KERNEL_KINDS; ++k) {
    if (ms) ms[k] = 0.0;
    if (launches) launches[k] = 0;
  }
  for (size_t i = 0; i < g_prof.used; i += 2) {
    TRY(cudaEventSynchronize(g_prof.ev[i + 1]));
    float t = 0.f;
    TRY(cudaEventElapsedTime(&t, g_prof.ev[i], g_prof.ev[i + 1]));
    const int k = g_prof.kind[i / 2];
    if (ms) ms[k] += t;
    if (launches) launches[k] += 1;
  }
  return TP_OK;
}

const char* tp_kernel_name(int kind) {
  static const char* names[TP_KERNEL_KINDS] = {"stencil_step", "imaging_sweep", "probe_gemm_tcgen05",
                                               "point_inject_sample", "reduce_fp64", "setup_other",
                                               "step_imaging_fused"};
  return (kind >= 0 && kind < TP_KERNEL_KINDS) ? names[kind] : "unknown";
}

}  // extern "C"
