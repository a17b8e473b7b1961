// C ABI of liblbm.so (declarations and contracts in include/lbm.h).
//
// Host side of one lattice: workspace carving, argument checks, the
// step loop replayed from captured CUDA graphs, the observable pipeline
// (point pass -> field pass -> finalize, all on the context stream), the
// convergence loop of Sec. IV, population transfer, checkpoints, the tile
// autotuner and the Tolman least-squares fit.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "lbm.h"
#include "lbm_launch.h"

using namespace lbm;

struct lbm_ctx {
  lbm_box box;
  double tau, G;
  lbm_eos eos;
  int stencil, prec;
  cudaStream_t stream;        // caller's stream (all work)
  cudaStream_t cap_stream;    // private stream used only to capture graphs
  char* ws;
  size_t ws_bytes;
  void* pop[2];
  void* u_old;
  FieldPartial* partials;
  long long max_partials;
  PointOut* pts;
  double* dP_prev;
  lbm_obs* obs_dev;
  int* err_dev;               // set by a kernel whose bounded wait ran out
  double* n_line;
  double* PT_line;
  double* PN_line;
  int line_len;
  int cur;                    // buffer holding the current state
  long long steps;
  int have_u_old;
  int initialised;
  double contrast0;
  double n0, scale;
  TileCfg step_cfg;
  int obs_zchunk;
  cudaGraphExec_t graph[2];   // graph_len steps, captured from parity 0 / 1
  int graph_len;
  lbm_obs last;
  int have_last;
  TmaMaps tma;                // tensor maps of pop[0] / pop[1] for the TMA step kernel (kind 7)
  char err[512];
};

// Named ranges on a profiler's timeline around the calls that drive the device
// (NVTX; without a tool attached each is a null check).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

namespace {

thread_local char g_err[512];

lbm_status fail(lbm_ctx* c, lbm_status s, const char* fmt, ...) {
  char* buf = c ? c->err : g_err;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, 512, fmt, ap);
  va_end(ap);
  return s;
}

}  // namespace

namespace lbm {
// error message of a call that has no context (read with lbm_last_error(NULL))
void set_global_error(const char* msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }
}  // namespace lbm

namespace {

#define LBM_CUDA(ctx, call)                                                              \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail((ctx), LBM_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));     \
  } while (0)

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

size_t storage_bytes(int prec) { return prec == kF64 ? 8 : (prec == kF32 ? 4 : 2); }

int radius_of(int stencil) { return stencil == 4 ? 1 : 2; }

bool valid_stencil(int s) { return s == 4 || s == 6 || s == 8; }
bool valid_prec(int p) { return p == kF64 || p == kF32 || p == kF16; }

constexpr int kObsBX = 32, kObsBY = 4;

int default_obs_zchunk(lbm_box b) { return b.nz < 8 ? b.nz : 8; }

long long obs_partials(lbm_box b, int zchunk) {
  return (long long)((b.nx + kObsBX - 1) / kObsBX) * ((b.ny + kObsBY - 1) / kObsBY) *
         ((b.nz + zchunk - 1) / zchunk);
}

constexpr size_t kStateDP = 64;     // offsets inside the state block
constexpr size_t kStateErr = 96;
constexpr size_t kStateObs = 128;
static_assert(sizeof(PointOut) <= kStateDP, "PointOut overlaps dP_prev");

struct Layout {
  size_t pop, u_old, partials, state, lines, total;
  long long npart;
};

Layout layout_of(lbm_box b, int prec) {
  Layout L;
  const size_t N = (size_t)b.nx * b.ny * b.nz;
  L.npart = obs_partials(b, default_obs_zchunk(b));
  L.pop = align256((size_t)Q * N * storage_bytes(prec));
  L.u_old = align256(3 * N * (prec == kF64 ? 8 : 4));
  L.partials = align256((size_t)L.npart * sizeof(FieldPartial));
  // state block: PointOut at 0, dP_prev at kStateDP, the lbm_obs record at kStateObs
  L.state = align256(kStateObs + sizeof(lbm_obs));
  L.lines = align256(3 * sizeof(double) * (size_t)(b.nx / 2 + 1));
  L.total = 2 * L.pop + L.u_old + L.partials + L.state + L.lines;
  return L;
}

bool box_ok(lbm_box b, int stencil) {
  const int m = 2 * radius_of(stencil) + 1;
  if (b.nx < m || b.ny < m || b.nz < m) return false;
  // node offsets inside one population plane are 32-bit in the kernels
  const double n = (double)b.nx * b.ny * b.nz;
  return n < 2147483647.0;
}

LatticeDesc desc_of(const lbm_ctx* c, int src_buf) {
  LatticeDesc d;
  d.src = c->pop[src_buf];
  d.dst = c->pop[src_buf ^ 1];
  d.nx = c->box.nx;
  d.ny = c->box.ny;
  d.nz = c->box.nz;
  d.plane = (long long)c->box.nx * c->box.ny * c->box.nz;
  d.omega = 1.0 / c->tau;
  d.n0 = c->n0;
  d.scale = c->scale;
  d.eos.kind = c->eos.kind;
  d.eos.G = c->G;
  d.eos.a = c->eos.a;
  d.eos.b = c->eos.b;
  d.eos.Rgas = c->eos.Rgas;
  d.eos.T = c->eos.T;
  d.err = c->err_dev;
  d.tma = c->tma.ok ? &c->tma : nullptr;
  set_float_params(d);
  return d;
}

// the TMA kernel (kind 7) as the default where it applies (else it is offered to the
// autotuner and lbm_set_tile only)
constexpr bool kTmaDefault = false;

TileCfg default_tile(lbm_box b, int prec, int stencil, double tau, bool allow_tma = true) {
  TileCfg t;
  // FP32 E4 at tau = 1 on boxes the TMA kernel takes: the moment kernel fed by
  // tensor-tile copies (kind 7)
  if (kTmaDefault && allow_tma && prec == kF32 && stencil == 4 && tau == 1.0 && tma_box_ok(b.nx, b.ny, b.nz, 8)) {
    t.kind = 7;
    t.bx = 32;
    t.by = 8;
    t.zchunk = 0;
    t.depth = 1;
    return t;
  }
  t.zchunk = b.nz < 16 ? b.nz : 16;
  t.bx = 32;
  t.by = stencil == 4 ? 8 : 4;
  if (prec == kF16) {
    // the moment kernel with FP16 staging (E4, tau = 1, nx % 8 == 0, nx >= 48),
    // else the register-load kernel
    if (stencil == 4 && tau == 1.0 && b.nx % 8 == 0 && b.nx >= 48) {
      t.kind = 5;
      t.zchunk = 0;
      t.depth = 2;
    }
    return t;
  }
  const int R = stencil == 4 ? 1 : 2;
  // the moment kernel (tau = 1; the chunked kernel otherwise) when the rows split
  // into 16-byte chunks: 32 x 8 tiles for E4 (prefetch depth 2 from 4M nodes on in
  // FP32: measured 3-6% faster there, 7% slower at 128^3), 32 x 4 for the wider
  // stencils, provided both kernels fit one CTA
  if (b.nx % 4 == 0 && b.nx >= 40) {
    const int by = stencil == 4 ? 8 : 4;
    const long long nodes = (long long)b.nx * b.ny * b.nz;
    const int depth = (prec == kF32 && stencil == 4 && nodes >= 4000000) ? 2 : 1;
    if (chunk_smem_bytes(prec == kF64 ? 8 : 4, R, 32, by, depth) <= kMaxSmemPerCta) {
      t.kind = 5;
      t.bx = 32;
      t.by = by;
      t.zchunk = 0;
      t.depth = depth;
      return t;
    }
  }
  // odd or narrow rows: the moment kernel with element copies (tau = 1; the
  // pipelined kernel otherwise) where two CTAs of it fit an SM
  {
    const int by = stencil == 4 ? 8 : 4;
    const size_t el = prec == kF64 ? 8 : 4;
    if (moment_elem_two_per_sm(el, R, 32, by, 1) && async_smem_bytes(el, R, 32, by, 1) <= kMaxSmemPerCta) {
      t.kind = 6;
      t.bx = 32;
      t.by = by;
      t.zchunk = 0;
      t.depth = 1;
      return t;
    }
  }
  // pipelined kernel with a launcher-chosen z chunk, if one compiled shape fits
  const int by_pref[2] = {(prec == kF64 || stencil != 4) ? 4 : 8, 4};
  for (int by : by_pref) {
    if (async_smem_bytes(prec == kF64 ? 8 : 4, R, 32, by, 1) <= kMaxSmemPerCta) {
      t.kind = 1;
      t.zchunk = 0;
      t.by = by;
      t.depth = 1;
      return t;
    }
  }
  return t;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to libcuda)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn tensor_map_encoder() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

long long tile_code(const TileCfg& t) {
  return (long long)t.kind * 100000000 + (long long)t.bx * 1000000 + t.by * 10000 +
         (t.kind >= 1 ? t.zchunk * 10 + t.depth : t.zchunk);
}

// every step configuration compiled for this precision and stencil
std::vector<TileCfg> step_candidates(const lbm_ctx* c) {
  std::vector<TileCfg> out;
  const int (*shapes)[2] = c->stencil == 4 ? kShapesE4 : kShapesWide;
  const int ns = c->stencil == 4 ? kNumShapesE4 : kNumShapesWide;
  const int zcands[] = {4, 8, 16, 32, 64};
  for (int k = 0; k < ns; ++k)
    for (int zc : zcands) {
      if (zc > c->box.nz && zc != 4) continue;
      TileCfg t{shapes[k][0], shapes[k][1], zc < c->box.nz ? zc : c->box.nz};
      out.push_back(t);
    }
  if (c->prec == kF16 && c->stencil == 4 && c->tau == 1.0 && c->box.nx % 8 == 0 && c->box.nx >= 48) {
    for (int depth : {1, 2})
      for (int zc : {0, 8, 16, 32}) {
        if (zc > c->box.nz) continue;
        TileCfg t{32, 8, zc};
        t.kind = 5;
        t.depth = depth;
        out.push_back(t);
      }
  }
  if (c->prec != kF16) {
    const int R = radius_of(c->stencil);
    if (c->tma.ok) {   // kind 7: the moment kernel fed by TMA tensor-tile copies
      for (int zc : {0, 8, 16, 32}) {
        if (zc > c->box.nz) continue;
        TileCfg t{c->tma.bx, c->tma.by, zc};
        t.kind = 7;
        t.depth = 1;
        out.push_back(t);
      }
    }
    {  // kind 6: the moment kernel with element copies (any nx), 2 CTAs per SM
      const int es[3][3] = {{32, 8, 1}, {32, 8, 2}, {32, 4, 1}};
      for (const auto& e : es) {
        if ((c->stencil == 4) != (e[1] == 8)) continue;
        if (async_smem_bytes(storage_bytes(c->prec), R, e[0], e[1], e[2]) > kMaxSmemPerCta) continue;
        if (!moment_elem_two_per_sm(storage_bytes(c->prec), R, e[0], e[1], e[2])) continue;
        for (int zc : {0, 8, 16, 32}) {
          if (zc > c->box.nz) continue;
          TileCfg t{e[0], e[1], zc};
          t.kind = 6;
          t.depth = e[2];
          out.push_back(t);
        }
      }
    }
    const int (*ms)[3] = c->stencil == 4 ? kMomentE4 : kMomentWide;
    const int nm = c->stencil == 4 ? kNumMomentE4 : kNumMomentWide;
    for (int k = 0; k < nm; ++k) {
      // the chunked kernel's requirements; both it and the chunked fallback must fit
      if (c->box.nx % 4 != 0 || c->box.nx < ms[k][0] + 8) continue;
      if (chunk_smem_bytes(storage_bytes(c->prec), R, ms[k][0], ms[k][1], ms[k][2]) > kMaxSmemPerCta)
        continue;
      for (int zc : {0, 8, 16, 32}) {
        if (zc > c->box.nz) continue;
        TileCfg t{ms[k][0], ms[k][1], zc};
        t.kind = 5;
        t.depth = ms[k][2];
        out.push_back(t);
      }
    }
    const int (*cs)[3] = c->stencil == 4 ? kChunkE4 : kChunkWide;
    const int nc = c->stencil == 4 ? kNumChunkE4 : kNumChunkWide;
    for (int k = 0; k < nc; ++k) {
      // 16-byte chunks of whole rows: nx % 4 == 0, and a staged row wraps at most once
      if (c->box.nx % 4 != 0 || c->box.nx < cs[k][0] + 8) continue;
      if (chunk_smem_bytes(storage_bytes(c->prec), R, cs[k][0], cs[k][1], cs[k][2]) > kMaxSmemPerCta)
        continue;
      for (int zc : {0, 8, 16, 32}) {
        if (zc > c->box.nz) continue;
        TileCfg t{cs[k][0], cs[k][1], zc};
        t.kind = 4;
        t.depth = cs[k][2];
        out.push_back(t);
      }
    }
    const int (*as)[3] = c->stencil == 4 ? kAsyncE4 : kAsyncWide;
    const int na = c->stencil == 4 ? kNumAsyncE4 : kNumAsyncWide;
    for (int k = 0; k < na; ++k) {
      // skip what does not fit one CTA's shared memory
      if (async_smem_bytes(storage_bytes(c->prec), R, as[k][0], as[k][1], as[k][2]) > kMaxSmemPerCta)
        continue;
      for (int zc : {0, 8, 16, 32}) {   // 0: the launcher's own choice
        if (zc > c->box.nz) continue;
        TileCfg t{as[k][0], as[k][1], zc};
        t.kind = 1;
        t.depth = as[k][2];
        out.push_back(t);
      }
    }
  }
  return out;
}

void drop_graphs(lbm_ctx* c) {
  for (int p = 0; p < 2; ++p) {
    if (c->graph[p]) cudaGraphExecDestroy(c->graph[p]);
    c->graph[p] = nullptr;
  }
}

lbm_status prepare_kernels(lbm_ctx* c) {
  // set the dynamic shared-memory limit of every kernel this context can use,
  // outside any stream capture
  LatticeDesc d = desc_of(c, 0);
  ObsArgs oa{};
  for (const TileCfg& t : step_candidates(c)) {
    TileCfg p = t;
    p.prepare = true;
    LBM_CUDA(c, launch_lattice(c->prec, c->stencil, kModeStep, d, p, oa, c->stream));
  }
  TileCfg t{kObsBX, kObsBY, 0};
  t.prepare = true;
  LBM_CUDA(c, launch_lattice(c->prec, c->stencil, kModeObs, d, t, oa, c->stream));
  return LBM_OK;
}

lbm_status launch_steps_eager(lbm_ctx* c, long long n, cudaStream_t s) {
  ObsArgs oa{};
  for (long long k = 0; k < n; ++k) {
    LatticeDesc d = desc_of(c, c->cur);
    LBM_CUDA(c, launch_lattice(c->prec, c->stencil, kModeStep, d, c->step_cfg, oa, s));
    c->cur ^= 1;
  }
  return LBM_OK;
}

lbm_status ensure_graph(lbm_ctx* c) {
  const int p = c->cur;
  if (c->graph[p]) return LBM_OK;
  cudaGraph_t g = nullptr;
  LBM_CUDA(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
  const int cur0 = c->cur;
  lbm_status st = launch_steps_eager(c, c->graph_len, c->cap_stream);
  c->cur = cur0;   // graph_len is even; capture does not advance the state
  cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
  if (st != LBM_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return fail(c, LBM_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&c->graph[p], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    c->graph[p] = nullptr;
    return fail(c, LBM_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
  }
  return LBM_OK;
}

lbm_status observe(lbm_ctx* c, double* rho_out, double* u_out, int write_u_old, bool finalize) {
  LatticeDesc d = desc_of(c, c->cur);
  LBM_CUDA(c, launch_point_obs(c->prec, c->stencil, d, c->pts, c->n_line, c->PT_line, c->PN_line,
                               c->stream));
  ObsArgs oa;
  oa.n_out = &c->pts->n_out;
  oa.u_old = c->u_old;
  oa.have_u_old = c->have_u_old;
  oa.partials = c->partials;
  oa.rho_out = rho_out;
  oa.u_out = u_out;
  oa.write_u_old = write_u_old;
  TileCfg t{kObsBX, kObsBY, c->obs_zchunk};
  LBM_CUDA(c, launch_lattice(c->prec, c->stencil, kModeObs, d, t, oa, c->stream));
  if (finalize) {
    FinalizeArgs fa;
    fa.partials = c->partials;
    fa.n_partials = lattice_grid_ctas(d, t);
    fa.pts = c->pts;
    fa.PT_line = c->PT_line;
    fa.line_len = c->line_len;
    fa.volume = d.plane;
    fa.contrast0 = c->contrast0;
    fa.center[0] = c->box.nx / 2;
    fa.center[1] = c->box.ny / 2;
    fa.center[2] = c->box.nz / 2;
    fa.have_u_old = c->have_u_old;
    fa.steps = c->steps;
    fa.dP_prev = c->dP_prev;
    fa.err = c->err_dev;
    fa.obs_out = c->obs_dev;
    LBM_CUDA(c, launch_finalize(fa, c->stream));
  }
  return LBM_OK;
}

lbm_status reset_history(lbm_ctx* c) {
  const double nan = NAN;
  LBM_CUDA(c, cudaMemcpyAsync(c->dP_prev, &nan, sizeof(double), cudaMemcpyHostToDevice, c->stream));
  LBM_CUDA(c, cudaMemsetAsync(c->err_dev, 0, sizeof(int), c->stream));
  LBM_CUDA(c, cudaStreamSynchronize(c->stream));
  c->have_u_old = 0;
  c->have_last = 0;
  c->steps = 0;
  c->initialised = 1;
  return LBM_OK;
}

void choose_storage(lbm_ctx* c, double n0, double maxdev) {
  if (c->prec == kF64) {
    c->n0 = 0.0;
    c->scale = 1.0;
    return;
  }
  c->n0 = n0;
  c->scale = 1.0;
  if (c->prec == kF16) {
    // power of two putting the largest expected |f_i - w_i n0| near 2^13
    // (half's largest normal number is 65504)
    const double m = maxdev > 0 ? maxdev : 1.0;
    int k = (int)floor(log2(8192.0 / m));
    if (k > 24) k = 24;
    if (k < -24) k = -24;
    c->scale = ldexp(1.0, k);
  }
}

double* temp_doubles(lbm_ctx* c) { return static_cast<double*>(c->pop[c->cur ^ 1]); }

#define LBM_CHECK_CTX(c)                                                  \
  do {                                                                    \
    if (!(c)) return fail(nullptr, LBM_EINVAL, "null context");           \
  } while (0)
#define LBM_CHECK_INIT(c)                                                                   \
  do {                                                                                      \
    if (!(c)->initialised) return fail((c), LBM_EINVAL, "field not initialised");          \
  } while (0)

}  // namespace

extern "C" {

size_t lbm_workspace_bytes(lbm_box box, int stencil, int prec) {
  if (!valid_stencil(stencil) || !valid_prec(prec) || !box_ok(box, stencil)) return 0;
  return layout_of(box, prec).total;
}

lbm_status lbm_create(lbm_box box, double tau, double G, lbm_eos eos, int stencil, int prec,
                      void* dev_workspace, size_t bytes, void* cuda_stream, lbm_ctx** out) {
  if (!out) return fail(nullptr, LBM_EINVAL, "out is null");
  *out = nullptr;
  if (!valid_stencil(stencil)) return fail(nullptr, LBM_EINVAL, "stencil must be 4, 6 or 8");
  if (!valid_prec(prec)) return fail(nullptr, LBM_EINVAL, "prec must be 0, 1 or 2");
  if (!box_ok(box, stencil))
    return fail(nullptr, LBM_EINVAL, "box %dx%dx%d not allowed (sides >= %d, below 2^31 nodes)", box.nx, box.ny, box.nz,
                2 * radius_of(stencil) + 1);
  if (!(tau > 0.5) || !isfinite(tau)) return fail(nullptr, LBM_EINVAL, "tau must be > 1/2");
  if (!isfinite(G)) return fail(nullptr, LBM_EINVAL, "G must be finite");
  if (eos.kind == LBM_PSI_EXP_INV) {
    const double Gc = -exp(2.0);   // psi = exp(-1/n): n_c = 1, G_c = -e^2
    if (!(G < Gc))
      return fail(nullptr, LBM_EINVAL, "G = %g is not below G_c = %.6f for psi = exp(-1/n): no coexistence",
                  G, Gc);
  } else if (eos.kind == LBM_PSI_ONE_MINUS_EXP) {
    if (!(G < -4.0))
      return fail(nullptr, LBM_EINVAL, "G = %g is not below G_c = -4 for psi = 1 - exp(-n): no coexistence", G);
  } else if (eos.kind == LBM_PSI_CS) {
    if (!(G < 0) || !(eos.T > 0) || !(eos.a > 0) || !(eos.b > 0) || !(eos.Rgas > 0))
      return fail(nullptr, LBM_EINVAL, "Carnahan-Starling psi needs G < 0 and a, b, Rgas, T > 0");
  } else {
    return fail(nullptr, LBM_EINVAL, "unknown psi kind %d", eos.kind);
  }
  const Layout L = layout_of(box, prec);
  if (!dev_workspace) return fail(nullptr, LBM_EINVAL, "workspace is null");
  if (((uintptr_t)dev_workspace & 255) != 0) return fail(nullptr, LBM_EINVAL, "workspace not 256-byte aligned");
  if (bytes < L.total)
    return fail(nullptr, LBM_ENOMEM, "workspace has %zu bytes, needs %zu", bytes, L.total);

  lbm_ctx* c = new lbm_ctx();
  memset(c->err, 0, sizeof(c->err));
  c->box = box;
  c->tau = tau;
  c->G = G;
  c->eos = eos;
  c->stencil = stencil;
  c->prec = prec;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  c->ws = static_cast<char*>(dev_workspace);
  c->ws_bytes = bytes;
  char* p = c->ws;
  c->pop[0] = p; p += L.pop;
  c->pop[1] = p; p += L.pop;
  c->u_old = p; p += L.u_old;
  c->partials = reinterpret_cast<FieldPartial*>(p); p += L.partials;
  c->max_partials = L.npart;
  c->pts = reinterpret_cast<PointOut*>(p);
  c->dP_prev = reinterpret_cast<double*>(p + kStateDP);
  c->obs_dev = reinterpret_cast<lbm_obs*>(p + kStateObs);
  c->err_dev = reinterpret_cast<int*>(p + kStateErr);
  p += L.state;
  c->line_len = box.nx / 2 + 1;
  c->n_line = reinterpret_cast<double*>(p);
  c->PT_line = c->n_line + c->line_len;
  c->PN_line = c->PT_line + c->line_len;
  c->cur = 0;
  c->n0 = 0.0;
  c->scale = 1.0;
  c->step_cfg = default_tile(box, prec, stencil, tau);
  if (prec == kF32 && stencil == 4 && tau == 1.0 && tma_box_ok(box.nx, box.ny, box.nz, 8))
    build_tma_maps(&c->tma, c->pop[0], c->pop[1], box.nx, box.ny, box.nz, 1, 32, 8);
  if (!c->tma.ok && c->step_cfg.kind == 7) c->step_cfg = default_tile(box, prec, stencil, tau, false);
  c->obs_zchunk = default_obs_zchunk(box);
  c->graph[0] = c->graph[1] = nullptr;
  c->graph_len = 128;
  cudaError_t e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete c;
    return fail(nullptr, LBM_ECUDA, "cudaStreamCreate failed: %s", cudaGetErrorString(e));
  }
  lbm_status st = prepare_kernels(c);
  if (st != LBM_OK) {
    snprintf(g_err, sizeof(g_err), "%s", c->err);
    cudaStreamDestroy(c->cap_stream);
    delete c;
    return st;
  }
  *out = c;
  return LBM_OK;
}

void lbm_destroy(lbm_ctx* c) {
  if (!c) return;
  drop_graphs(c);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  delete c;
}

lbm_status lbm_init_drop(lbm_ctx* c, const double center[3], double R, double rho_in,
                         double rho_out, double width) {
  LBM_CHECK_CTX(c);
  if (!center) return fail(c, LBM_EINVAL, "center is null");
  if (!(R > 0) || !(width > 0) || !(rho_in > 0) || !(rho_out > 0) || !isfinite(R) ||
      !isfinite(rho_in) || !isfinite(rho_out) || !isfinite(width))
    return fail(c, LBM_EINVAL, "R, width and densities must be positive and finite");
  for (int k = 0; k < 3; ++k)
    if (!isfinite(center[k])) return fail(c, LBM_EINVAL, "center must be finite");
  // shift: the mean density of a sharp sphere of radius R in the box, so that
  // the phase filling most of the volume is stored with the smallest values
  const double V = (double)c->box.nx * c->box.ny * c->box.nz;
  const double frac = fmin(1.0, 4.0 * M_PI * R * R * R / (3.0 * V));
  const double mean = rho_out + (rho_in - rho_out) * frac;
  choose_storage(c, mean, (1.0 / 3.0) * fmax(fabs(rho_in - mean), fabs(rho_out - mean)));
  c->cur = 0;
  drop_graphs(c);
  DropInit di{center[0], center[1], center[2], R, rho_in, rho_out, width};
  LatticeDesc d = desc_of(c, 1);   // writes pop[0]
  LBM_CUDA(c, launch_init_drop(c->prec, d, di, c->stream));
  c->contrast0 = fabs(rho_in - rho_out);
  return reset_history(c);
}

lbm_status lbm_init_rho(lbm_ctx* c, const double* host_rho) {
  LBM_CHECK_CTX(c);
  if (!host_rho) return fail(c, LBM_EINVAL, "host_rho is null");
  const long long N = (long long)c->box.nx * c->box.ny * c->box.nz;
  double mn = host_rho[0], mx = host_rho[0], sum = 0.0;
  for (long long k = 0; k < N; ++k) {
    const double v = host_rho[k];
    if (!(v > 0) || !isfinite(v)) return fail(c, LBM_EINVAL, "density must be positive and finite");
    mn = v < mn ? v : mn;
    mx = v > mx ? v : mx;
    sum += v;
  }
  const double mean = sum / (double)N;
  choose_storage(c, mean, (1.0 / 3.0) * fmax(mx - mean, mean - mn));
  c->cur = 0;
  drop_graphs(c);
  double* tmp = static_cast<double*>(c->pop[1]);
  LBM_CUDA(c, cudaMemcpyAsync(tmp, host_rho, N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  LatticeDesc d = desc_of(c, 1);   // writes pop[0]
  LBM_CUDA(c, launch_init_rho(c->prec, d, tmp, c->stream));
  c->contrast0 = mx - mn;
  return reset_history(c);
}

lbm_status lbm_set_populations(lbm_ctx* c, const double* host_f) {
  LBM_CHECK_CTX(c);
  if (!host_f) return fail(c, LBM_EINVAL, "host_f is null");
  const long long N = (long long)c->box.nx * c->box.ny * c->box.nz;
  std::vector<double> n(N, 0.0);
  for (int i = 0; i < Q; ++i)
    for (long long k = 0; k < N; ++k) {
      const double v = host_f[(long long)i * N + k];
      if (!isfinite(v)) return fail(c, LBM_EINVAL, "populations must be finite");
      n[k] += v;
    }
  double mn = n[0], mx = n[0], sum = 0.0;
  for (long long k = 0; k < N; ++k) {
    mn = n[k] < mn ? n[k] : mn;
    mx = n[k] > mx ? n[k] : mx;
    sum += n[k];
  }
  const double mean = sum / (double)N;
  double maxdev = 0.0;
  for (int i = 0; i < Q; ++i)
    for (long long k = 0; k < N; ++k)
      maxdev = fmax(maxdev, fabs(host_f[(long long)i * N + k] - wq(i) * mean));
  choose_storage(c, mean, maxdev);
  c->cur = 0;
  drop_graphs(c);
  double* tmp = static_cast<double*>(c->pop[1]);
  LatticeDesc d = desc_of(c, 1);   // writes pop[0]
  for (int i = 0; i < Q; ++i) {
    LBM_CUDA(c, cudaMemcpyAsync(tmp, host_f + (long long)i * N, N * sizeof(double),
                                cudaMemcpyHostToDevice, c->stream));
    LBM_CUDA(c, launch_set_plane(c->prec, d, i, tmp, c->stream));
  }
  c->contrast0 = mx - mn;
  return reset_history(c);
}

lbm_status lbm_get_populations(lbm_ctx* c, double* host_f) {
  LBM_CHECK_CTX(c);
  LBM_CHECK_INIT(c);
  if (!host_f) return fail(c, LBM_EINVAL, "host_f is null");
  const long long N = (long long)c->box.nx * c->box.ny * c->box.nz;
  double* tmp = temp_doubles(c);
  LatticeDesc d = desc_of(c, c->cur);
  for (int i = 0; i < Q; ++i) {
    LBM_CUDA(c, launch_get_plane(c->prec, d, i, tmp, c->stream));
    LBM_CUDA(c, cudaMemcpyAsync(host_f + (long long)i * N, tmp, N * sizeof(double),
                                cudaMemcpyDeviceToHost, c->stream));
  }
  LBM_CUDA(c, cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

lbm_status lbm_step(lbm_ctx* c, long long n) {
  NvtxRange nvtx("lbm_step");
  LBM_CHECK_CTX(c);
  LBM_CHECK_INIT(c);
  if (n < 0) return fail(c, LBM_EINVAL, "n must be >= 0");
  while (n >= c->graph_len) {
    lbm_status st = ensure_graph(c);
    if (st != LBM_OK) return st;
    LBM_CUDA(c, cudaGraphLaunch(c->graph[c->cur], c->stream));
    n -= c->graph_len;
    c->steps += c->graph_len;
  }
  lbm_status st = launch_steps_eager(c, n, c->stream);
  if (st != LBM_OK) return st;
  c->steps += n;
  return LBM_OK;
}

lbm_status lbm_observables(lbm_ctx* c, lbm_obs* out) {
  NvtxRange nvtx("lbm_observables");
  LBM_CHECK_CTX(c);
  LBM_CHECK_INIT(c);
  lbm_status st = observe(c, nullptr, nullptr, 1, true);
  if (st != LBM_OK) return st;
  LBM_CUDA(c, cudaMemcpyAsync(&c->last, c->obs_dev, sizeof(lbm_obs), cudaMemcpyDeviceToHost, c->stream));
  LBM_CUDA(c, cudaStreamSynchronize(c->stream));
  c->have_u_old = 1;
  c->have_last = 1;
  if (out) *out = c->last;
  return LBM_OK;
}

lbm_status lbm_run_to_convergence(lbm_ctx* c, long long max_steps, long long check_every,
                                  double tol_dP_rel, double tol_du, long long* steps_done,
                                  int* criterion) {
  NvtxRange nvtx("lbm_run_to_convergence");
  LBM_CHECK_CTX(c);
  LBM_CHECK_INIT(c);
  if (max_steps < 0 || check_every < 1) return fail(c, LBM_EINVAL, "max_steps >= 0, check_every >= 1");
  lbm_status st;
  if (!c->have_last) {
    st = lbm_observables(c, nullptr);
    if (st != LBM_OK) return st;
  }
  long long done = 0;
  int crit = 0;
  while (done < max_steps) {
    const long long k = (max_steps - done < check_every) ? max_steps - done : check_every;
    st = lbm_step(c, k);
    if (st != LBM_OK) return st;
    done += k;
    const unsigned prev_bits = c->last.status_bits;
    st = lbm_observables(c, nullptr);
    if (st != LBM_OK) return st;
    if (c->last.status_bits & 16u) {
      if (steps_done) *steps_done = done;
      if (criterion) *criterion = 0;
      return fail(c, LBM_ETIMEOUT, "a step kernel's bounded wait for its copies ran out");
    }
    if (c->last.status_bits & 8u) {
      if (steps_done) *steps_done = done;
      if (criterion) *criterion = 0;
      return fail(c, LBM_ENUMERIC, "non-finite or non-positive density after %lld steps", c->steps);
    }
    if ((c->last.status_bits & 2u) && (prev_bits & 2u)) {   // collapsed at two checks in a row
      if (steps_done) *steps_done = done;
      if (criterion) *criterion = 0;
      c->last.criterion = 0;
      return fail(c, LBM_ECOLLAPSE, "the droplet/bubble collapsed (after %lld steps)", c->steps);
    }
    if (c->last.dP_rel_change < tol_dP_rel) { crit = 1; break; }
    if (c->last.du < tol_du) { crit = 2; break; }
  }
  c->last.criterion = crit;
  if (steps_done) *steps_done = done;
  if (criterion) *criterion = crit;
  if (!crit) return fail(c, LBM_ENOTCONV, "not converged after %lld steps", done);
  return LBM_OK;
}

lbm_status lbm_rho_profile(lbm_ctx* c, double* host_out, long long len) {
  LBM_CHECK_CTX(c);
  if (!host_out || len != c->line_len) return fail(c, LBM_EINVAL, "len must be nx/2 + 1 = %d", c->line_len);
  if (!c->have_last) return fail(c, LBM_EINVAL, "call lbm_observables first");
  LBM_CUDA(c, cudaMemcpyAsync(host_out, c->n_line, len * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  LBM_CUDA(c, cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

lbm_status lbm_pt_profile(lbm_ctx* c, double* host_out, long long len) {
  LBM_CHECK_CTX(c);
  if (!host_out || len != c->line_len) return fail(c, LBM_EINVAL, "len must be nx/2 + 1 = %d", c->line_len);
  if (!c->have_last) return fail(c, LBM_EINVAL, "call lbm_observables first");
  LBM_CUDA(c, cudaMemcpyAsync(host_out, c->PT_line, len * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  LBM_CUDA(c, cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

lbm_status lbm_pn_profile(lbm_ctx* c, double* host_out, long long len) {
  LBM_CHECK_CTX(c);
  if (!host_out || len != c->line_len) return fail(c, LBM_EINVAL, "len must be nx/2 + 1 = %d", c->line_len);
  if (!c->have_last) return fail(c, LBM_EINVAL, "call lbm_observables first");
  LBM_CUDA(c, cudaMemcpyAsync(host_out, c->PN_line, len * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  LBM_CUDA(c, cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

size_t lbm_flat_workspace_bytes(int Lx, int stencil, int prec) {
  if (!valid_stencil(stencil)) return 0;
  const int m = 2 * radius_of(stencil) + 1;
  return lbm_workspace_bytes(lbm_box{Lx, m, m}, stencil, prec);
}

lbm_status lbm_flat_interface(double tau, double G, lbm_eos eos, int stencil, int prec, int Lx,
                              double rho_l0, double rho_g0, long long max_steps, double tol_du,
                              void* dev_workspace, size_t bytes, void* cuda_stream, double* n_g,
                              double* n_l, double* sigma0, long long* steps) {
  if (!n_g || !n_l || !sigma0) return fail(nullptr, LBM_EINVAL, "null output pointer");
  if (!valid_stencil(stencil)) return fail(nullptr, LBM_EINVAL, "stencil must be 4, 6 or 8");
  if (Lx < 8) return fail(nullptr, LBM_EINVAL, "Lx must be >= 8");
  if (rho_l0 == 0.0 && rho_g0 == 0.0) {   // start from the continuum coexistence
    const lbm_status e = lbm_coexistence_estimate(eos, G, &rho_g0, &rho_l0, nullptr);
    if (e != LBM_OK) return e;
  }
  if (!(rho_l0 > rho_g0) || !(rho_g0 > 0)) return fail(nullptr, LBM_EINVAL, "need rho_l0 > rho_g0 > 0");
  const int m = 2 * radius_of(stencil) + 1;
  const lbm_box box{Lx, m, m};
  lbm_ctx* c = nullptr;
  lbm_status st = lbm_create(box, tau, G, eos, stencil, prec, dev_workspace, bytes, cuda_stream, &c);
  if (st != LBM_OK) return st;
  // Eq. (24): liquid outside a gas strip of width Lx/2 centred at x0 = Lx/2
  std::vector<double> rho((size_t)Lx * m * m);
  const double x0 = 0.5 * Lx, w = 0.5 * Lx, a = 0.5 * (rho_l0 - rho_g0);
  for (int x = 0; x < Lx; ++x) {
    const double n = 0.5 * (rho_l0 + rho_g0) - a * tanh(x - (x0 - 0.5 * w)) +
                     a * (tanh(x - (x0 + 0.5 * w)) + 1.0);
    for (int k = 0; k < m * m; ++k) rho[(size_t)k * Lx + x] = n;
  }
  long long done = 0;
  int crit = 0;
  st = lbm_init_rho(c, rho.data());
  // the flat interface ends at rest: the delta-u test decides (Delta P is zero there)
  if (st == LBM_OK) st = lbm_run_to_convergence(c, max_steps, 2048, -1.0, tol_du, &done, &crit);
  if (st == LBM_OK || st == LBM_ENOTCONV) {
    const lbm_status keep = st;
    std::vector<double> pt(c->line_len), pn(c->line_len);
    st = lbm_pt_profile(c, pt.data(), c->line_len);
    if (st == LBM_OK) st = lbm_pn_profile(c, pn.data(), c->line_len);
    if (st == LBM_OK) {
      // Eq. (25) over [Lx/2, Lx]: from the gas centre to the liquid at the far edge
      double s = 0.0;
      for (int r = 0; r < c->line_len; ++r)
        s += ((r == 0 || r == c->line_len - 1) ? 0.5 : 1.0) * (pn[r] - pt[r]);
      *n_g = c->last.n_in;
      *n_l = c->last.n_out;
      *sigma0 = s;
      if (steps) *steps = done;
      st = keep;
    }
  }
  if (st != LBM_OK) snprintf(g_err, sizeof(g_err), "%s", c->err);
  lbm_destroy(c);
  return st;
}

lbm_status lbm_sigma_of_R(lbm_ctx* c, const double* R, double* sigma, double* dsigma, long long m) {
  LBM_CHECK_CTX(c);
  if (!c->have_last) return fail(c, LBM_EINVAL, "call lbm_observables first");
  if (m < 0 || (m > 0 && (!R || !sigma || !dsigma))) return fail(c, LBM_EINVAL, "bad arrays");
  const double dP = c->last.dP, C = c->last.C, D = c->last.D;
  for (long long k = 0; k < m; ++k) {
    if (!(R[k] > 0)) return fail(c, LBM_EINVAL, "R must be > 0");
    const double r = R[k];
    sigma[k] = dP * r / 3.0 + C / (r * r);
    dsigma[k] = dP / 3.0 - 2.0 * C / (r * r * r) + 2.0 * D / (r * r);
  }
  return LBM_OK;
}

lbm_status lbm_copy_rho(lbm_ctx* c, double* host_out) {
  LBM_CHECK_CTX(c);
  LBM_CHECK_INIT(c);
  if (!host_out) return fail(c, LBM_EINVAL, "host_out is null");
  const long long N = (long long)c->box.nx * c->box.ny * c->box.nz;
  double* tmp = temp_doubles(c);
  lbm_status st = observe(c, tmp, nullptr, 0, false);
  if (st != LBM_OK) return st;
  LBM_CUDA(c, cudaMemcpyAsync(host_out, tmp, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  LBM_CUDA(c, cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

lbm_status lbm_copy_velocity(lbm_ctx* c, double* host_out) {
  LBM_CHECK_CTX(c);
  LBM_CHECK_INIT(c);
  if (!host_out) return fail(c, LBM_EINVAL, "host_out is null");
  const long long N = (long long)c->box.nx * c->box.ny * c->box.nz;
  double* tmp = temp_doubles(c);
  lbm_status st = observe(c, nullptr, tmp, 0, false);
  if (st != LBM_OK) return st;
  LBM_CUDA(c, cudaMemcpyAsync(host_out, tmp, 3 * N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  LBM_CUDA(c, cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

static const char kMagic[8] = {'L', 'B', 'M', 'G', 'B', '3', '0', '0'};

struct CkptHeader {
  char magic[8];
  int version, nx, ny, nz, prec, stencil;
  long long steps;
  double n0, scale, contrast0;
};

lbm_status lbm_save(lbm_ctx* c, const char* path) {
  LBM_CHECK_CTX(c);
  LBM_CHECK_INIT(c);
  if (!path) return fail(c, LBM_EINVAL, "path is null");
  const size_t bytes = (size_t)Q * c->box.nx * c->box.ny * c->box.nz * storage_bytes(c->prec);
  std::vector<char> buf(bytes);
  LBM_CUDA(c, cudaMemcpyAsync(buf.data(), c->pop[c->cur], bytes, cudaMemcpyDeviceToHost, c->stream));
  LBM_CUDA(c, cudaStreamSynchronize(c->stream));
  FILE* f = fopen(path, "wb");
  if (!f) return fail(c, LBM_EINVAL, "cannot open %s for writing", path);
  CkptHeader h;
  memcpy(h.magic, kMagic, 8);
  h.version = 1;
  h.nx = c->box.nx; h.ny = c->box.ny; h.nz = c->box.nz;
  h.prec = c->prec; h.stencil = c->stencil;
  h.steps = c->steps; h.n0 = c->n0; h.scale = c->scale; h.contrast0 = c->contrast0;
  const bool ok = fwrite(&h, sizeof(h), 1, f) == 1 && fwrite(buf.data(), 1, bytes, f) == bytes;
  fclose(f);
  if (!ok) return fail(c, LBM_EINVAL, "short write to %s", path);
  return LBM_OK;
}

lbm_status lbm_load(lbm_ctx* c, const char* path) {
  LBM_CHECK_CTX(c);
  if (!path) return fail(c, LBM_EINVAL, "path is null");
  FILE* f = fopen(path, "rb");
  if (!f) return fail(c, LBM_EINVAL, "cannot open %s", path);
  CkptHeader h;
  if (fread(&h, sizeof(h), 1, f) != 1 || memcmp(h.magic, kMagic, 8) != 0 || h.version != 1) {
    fclose(f);
    return fail(c, LBM_EINVAL, "%s is not a checkpoint of this library", path);
  }
  if (h.nx != c->box.nx || h.ny != c->box.ny || h.nz != c->box.nz || h.prec != c->prec ||
      h.stencil != c->stencil) {
    fclose(f);
    return fail(c, LBM_EINVAL, "checkpoint box/precision/stencil differ from the context");
  }
  const size_t bytes = (size_t)Q * c->box.nx * c->box.ny * c->box.nz * storage_bytes(c->prec);
  std::vector<char> buf(bytes);
  const bool ok = fread(buf.data(), 1, bytes, f) == bytes;
  fclose(f);
  if (!ok) return fail(c, LBM_EINVAL, "truncated checkpoint %s", path);
  c->cur = 0;
  drop_graphs(c);
  LBM_CUDA(c, cudaMemcpyAsync(c->pop[0], buf.data(), bytes, cudaMemcpyHostToDevice, c->stream));
  c->n0 = h.n0;
  c->scale = h.scale;
  c->contrast0 = h.contrast0;
  lbm_status st = reset_history(c);
  c->steps = h.steps;
  return st;
}

lbm_status lbm_autotune(lbm_ctx* c, int reps, long long* choice) {
  LBM_CHECK_CTX(c);
  LBM_CHECK_INIT(c);
  if (reps < 2) reps = 2;
  reps += reps & 1;
  cudaEvent_t e0, e1;
  LBM_CUDA(c, cudaEventCreate(&e0));
  LBM_CUDA(c, cudaEventCreate(&e1));
  TileCfg best = c->step_cfg;
  float best_ms = 1e30f;
  lbm_status st = LBM_OK;
  for (const TileCfg& t : step_candidates(c)) {
    c->step_cfg = t;
    st = launch_steps_eager(c, 2, c->stream);
    if (st != LBM_OK) break;
    cudaEventRecord(e0, c->stream);
    st = launch_steps_eager(c, reps, c->stream);
    if (st != LBM_OK) break;
    cudaEventRecord(e1, c->stream);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) { st = fail(c, LBM_ECUDA, "autotune: %s", cudaGetErrorString(e)); break; }
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    c->steps += reps + 2;
    if (ms < best_ms) { best_ms = ms; best = t; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->step_cfg = best;
  drop_graphs(c);
  c->have_u_old = 0;
  if (st != LBM_OK) return st;
  if (choice) *choice = tile_code(best);
  return LBM_OK;
}

lbm_status lbm_set_tile(lbm_ctx* c, long long code) {
  LBM_CHECK_CTX(c);
  // code = kind 10^8 + bx 10^6 + by 10^4 + (kind ? zchunk 10 + depth : zchunk); any
  // z chunk in range is accepted for a compiled (kind, bx, by, depth)
  const int kind = (int)(code / 100000000), bx = (int)(code / 1000000 % 100), by = (int)(code / 10000 % 100);
  const int low = (int)(code % 10000);
  const int zc = kind >= 1 ? low / 10 : low, depth = kind >= 1 ? low % 10 : 1;
  const bool zc_ok = kind >= 1 ? (zc >= 0 && zc <= c->box.nz) : (zc >= 1 && zc <= c->box.nz);
  for (const TileCfg& t : step_candidates(c)) {
    if (zc_ok && t.kind == kind && t.bx == bx && t.by == by && (kind == 0 || t.depth == depth)) {
      TileCfg chosen = t;
      chosen.zchunk = zc;
      c->step_cfg = chosen;
      drop_graphs(c);
      return LBM_OK;
    }
  }
  return fail(c, LBM_EINVAL, "tile code %lld is not compiled for this precision/stencil/box", code);
}

lbm_status lbm_get_tile(const lbm_ctx* c, long long* code) {
  if (!c || !code) return fail(nullptr, LBM_EINVAL, "null argument");
  *code = tile_code(c->step_cfg);
  return LBM_OK;
}

lbm_status lbm_default_tile(lbm_box box, int stencil, int prec, double tau, long long* code) {
  if (!code) return fail(nullptr, LBM_EINVAL, "code is null");
  if (!valid_stencil(stencil)) return fail(nullptr, LBM_EINVAL, "stencil must be 4, 6 or 8");
  if (!valid_prec(prec)) return fail(nullptr, LBM_EINVAL, "prec must be 0, 1 or 2");
  if (!box_ok(box, stencil))
    return fail(nullptr, LBM_EINVAL, "box %dx%dx%d not allowed (sides >= %d, below 2^31 nodes)", box.nx, box.ny, box.nz,
                2 * radius_of(stencil) + 1);
  if (!(tau > 0.5) || !isfinite(tau)) return fail(nullptr, LBM_EINVAL, "tau must be > 1/2");
  *code = tile_code(default_tile(box, prec, stencil, tau));
  return LBM_OK;
}

lbm_status lbm_storage_params(const lbm_ctx* c, double* n0, double* scale) {
  if (!c) return fail(nullptr, LBM_EINVAL, "null context");
  if (n0) *n0 = c->n0;
  if (scale) *scale = c->scale;
  return LBM_OK;
}

const char* lbm_strerror(lbm_status s) {
  switch (s) {
    case LBM_OK: return "ok";
    case LBM_EINVAL: return "invalid argument";
    case LBM_ENOMEM: return "workspace too small";
    case LBM_ECUDA: return "CUDA error";
    case LBM_ENUMERIC: return "non-finite or non-positive density";
    case LBM_ENOTCONV: return "not converged";
    case LBM_ENOMIN: return "sigma[R] has no minimum";
    case LBM_ECOLLAPSE: return "droplet/bubble collapsed";
    case LBM_EOFFCENTER: return "centre of mass off centre";
    case LBM_ETIMEOUT: return "device wait timed out";
  }
  return "unknown status";
}

const char* lbm_last_error(const lbm_ctx* c) { return c ? c->err : g_err; }

// ---------------------------------------------------------------- continuum coexistence
// Bulk pressure of Eq. (10), P(n) = n c_s^2 + G c_s^2 psi(n)^2 / 2 (e_2 = 1), and
// the weight psi'(n) / psi(n) of the flat interface's mechanical-stability
// condition.  To leading order in gradients Eq. (9) gives, through a flat
// interface, P_N = P(n) + (G c_s^2 / 4) psi psi_xx; with P_N = p_0 constant,
// (p_0 - P) psi_x / psi = (G c_s^2 / 8) d(psi_x^2)/dx integrates to zero across
// the interface: int_{n_g}^{n_l} (p_0 - P(n)) psi'/psi dn = 0 with
// P(n_g) = P(n_l) = p_0 (an equal-area rule in the variable ln psi).

namespace {

struct HostEos {
  lbm_eos e;
  double G;
  double psi(double n) const {
    if (e.kind == LBM_PSI_EXP_INV) return exp(-1.0 / n);
    if (e.kind == LBM_PSI_ONE_MINUS_EXP) return -expm1(-n);
    return sqrt(2.0 * (p_cs(n) - n / 3.0) / (G / 3.0));
  }
  double p_cs(double n) const {   // Carnahan-Starling pressure
    const double q = 0.25 * e.b * n, om = 1.0 - q;
    return n * e.Rgas * e.T * (1.0 + q + q * q - q * q * q) / (om * om * om) - e.a * n * n;
  }
  double dp_cs(double n) const {  // d p_CS / dn
    const double q = 0.25 * e.b * n, om = 1.0 - q;
    return e.Rgas * e.T * (1.0 + 4.0 * q + 4.0 * q * q - 4.0 * q * q * q + q * q * q * q) /
               (om * om * om * om) - 2.0 * e.a * n;
  }
  double P(double n) const {
    if (e.kind == LBM_PSI_CS) return p_cs(n);   // the mapped psi returns p_CS exactly
    const double p = psi(n);
    return n / 3.0 + G / 6.0 * p * p;
  }
  double dP(double n) const {     // dP/dn = c_s^2 + G c_s^2 psi psi'
    if (e.kind == LBM_PSI_CS) return dp_cs(n);
    return 1.0 / 3.0 + G / 3.0 * psi(n) * dpsi(n);
  }
  double dpsi(double n) const {
    if (e.kind == LBM_PSI_EXP_INV) return exp(-1.0 / n) / (n * n);
    if (e.kind == LBM_PSI_ONE_MINUS_EXP) return exp(-n);
    return (dp_cs(n) - 1.0 / 3.0) / (G / 3.0 * psi(n));   // from psi^2 = 2 (p_CS - n/3)/(G/3)
  }
  double weight(double n) const { return dpsi(n) / psi(n); }
};

// root of P(n) = p on [a, b] where P is monotone, by bisection
double bisect_P(const HostEos& h, double p, double a, double b) {
  double fa = h.P(a) - p;
  for (int it = 0; it < 200 && b - a > 1e-15 * fabs(b); ++it) {
    const double m = 0.5 * (a + b), fm = h.P(m) - p;
    if ((fm < 0) == (fa < 0)) { a = m; fa = fm; } else { b = m; }
  }
  return 0.5 * (a + b);
}

// int_{ng}^{nl} (p0 - P(n)) psi'/psi dn: 5-point Gauss-Legendre on panels
// uniform in log n (the weight grows like 1/n as n -> 0 for psi = 1 - exp(-n))
double area(const HostEos& h, double p0, double ng, double nl) {
  static const double x[5] = {-0.9061798459386640, -0.5384693101056831, 0.0, 0.5384693101056831,
                              0.9061798459386640};
  static const double w[5] = {0.2369268850561891, 0.4786286704993665, 0.5688888888888889,
                              0.4786286704993665, 0.2369268850561891};
  const int panels = 768;
  const double a = log(ng), b = log(nl), hw = 0.5 * (b - a) / panels;
  double s = 0.0;
  for (int k = 0; k < panels; ++k) {
    const double mid = a + (2 * k + 1) * hw;
    for (int j = 0; j < 5; ++j) {
      const double n = exp(mid + hw * x[j]);
      s += w[j] * (p0 - h.P(n)) * h.weight(n) * n;
    }
  }
  return s * hw;
}

}  // namespace

lbm_status lbm_coexistence_estimate(lbm_eos eos, double G, double* n_g, double* n_l, double* p0) {
  if (!n_g || !n_l) return fail(nullptr, LBM_EINVAL, "null output pointer");
  if (!isfinite(G) || !(G < 0)) return fail(nullptr, LBM_EINVAL, "G must be negative");
  if (eos.kind != LBM_PSI_EXP_INV && eos.kind != LBM_PSI_ONE_MINUS_EXP && eos.kind != LBM_PSI_CS)
    return fail(nullptr, LBM_EINVAL, "unknown psi kind %d", eos.kind);
  if (eos.kind == LBM_PSI_CS && (!(eos.b > 0) || !(eos.T > 0) || !(eos.a > 0) || !(eos.Rgas > 0)))
    return fail(nullptr, LBM_EINVAL, "Carnahan-Starling psi needs a, b, Rgas, T > 0");
  const HostEos h{eos, G};
  const double lo = eos.kind == LBM_PSI_EXP_INV ? 0.02 : 1e-6;
  double hi = 4.0;
  if (eos.kind == LBM_PSI_CS) {
    // the mapped psi is real while p_CS(n) <= n c_s^2 (G < 0); stay below that density
    hi = 0.999 * 4.0 / eos.b;
    for (int k = 1; k <= 20000; ++k) {
      const double n = lo + (hi - lo) * k / 20000;
      if (h.p_cs(n) - n / 3.0 >= 0) { hi = lo + (hi - lo) * (k - 1) / 20000; break; }
    }
  }
  // spinodals: the first maximum of P (gas side) and the minimum after it (liquid side)
  const int M = 20000;
  double n_sg = -1, n_sl = -1;
  double prev = h.dP(lo);
  for (int k = 1; k <= M; ++k) {
    const double n = lo + (hi - lo) * k / M, d = h.dP(n);
    if (!isfinite(d)) continue;
    if (n_sg < 0 && prev > 0 && d <= 0) n_sg = n;
    else if (n_sg > 0 && prev < 0 && d >= 0) { n_sl = n; break; }
    prev = d;
  }
  if (n_sg < 0 || n_sl < 0)
    return fail(nullptr, LBM_EINVAL, "P(n) has no van der Waals loop in [%g, %g]: no coexistence", lo, hi);
  // bisection on n_g in (n_min, n_sg): p_0 = P(n_g), n_l the liquid root above n_sl
  const double p_floor = fmax(h.P(n_sl), h.P(lo));
  if (!(h.P(hi) > h.P(n_sg)))
    return fail(nullptr, LBM_EINVAL, "the liquid branch does not reach the gas spinodal pressure below n = %g", hi);
  double a = h.P(lo) >= p_floor ? lo : bisect_P(h, p_floor, lo, n_sg);
  double b = n_sg;
  a += 1e-12 * (b - a);
  b -= 1e-12 * (b - a);
  auto A = [&](double ng) {
    const double p = h.P(ng);
    return area(h, p, ng, bisect_P(h, p, n_sl, hi));
  };
  double fa = A(a);
  const double fb = A(b);
  if ((fa < 0) == (fb < 0))
    return fail(nullptr, LBM_EINVAL, "the equal-area condition has no root between the spinodals");
  for (int it = 0; it < 100 && b - a > 1e-15 * b; ++it) {
    const double m = 0.5 * (a + b), fm = A(m);
    if ((fm < 0) == (fa < 0)) { a = m; fa = fm; } else { b = m; }
  }
  const double ng = 0.5 * (a + b), p = h.P(ng);
  *n_g = ng;
  *n_l = bisect_P(h, p, n_sl, hi);
  if (p0) *p0 = p;
  return LBM_OK;
}

lbm_status lbm_tolman_fit(const double* R_s, const double* sigma_s, const int* is_bubble,
                          long long m, int quadratic, double* sigma0, double* delta, double* cc) {
  if (m < 0 || (m > 0 && (!R_s || !sigma_s || !is_bubble)) || !sigma0 || !delta || !cc)
    return fail(nullptr, LBM_EINVAL, "bad arguments");
  const int np = quadratic ? 3 : 2;
  // normal equations A^T A a = A^T s with rows (1, x, x^2), x = +-1/R_s
  double M[3][3] = {{0}}, v[3] = {0};
  long long used = 0;
  for (long long k = 0; k < m; ++k) {
    if (!isfinite(R_s[k]) || !isfinite(sigma_s[k]) || R_s[k] == 0.0) continue;
    const double x = (is_bubble[k] ? -1.0 : 1.0) / R_s[k];
    const double row[3] = {1.0, x, x * x};
    for (int i = 0; i < np; ++i) {
      v[i] += row[i] * sigma_s[k];
      for (int j = 0; j < np; ++j) M[i][j] += row[i] * row[j];
    }
    ++used;
  }
  if (used < np) return fail(nullptr, LBM_EINVAL, "need at least %d usable points, have %lld", np, used);
  // Gauss-Jordan with partial pivoting
  double a[3] = {0, 0, 0};
  for (int col = 0; col < np; ++col) {
    int piv = col;
    for (int r = col + 1; r < np; ++r)
      if (fabs(M[r][col]) > fabs(M[piv][col])) piv = r;
    if (M[piv][col] == 0.0) return fail(nullptr, LBM_EINVAL, "singular fit");
    if (piv != col) {
      for (int j = 0; j < np; ++j) { double t = M[col][j]; M[col][j] = M[piv][j]; M[piv][j] = t; }
      double t = v[col]; v[col] = v[piv]; v[piv] = t;
    }
    for (int r = 0; r < np; ++r) {
      if (r == col) continue;
      const double f = M[r][col] / M[col][col];
      for (int j = 0; j < np; ++j) M[r][j] -= f * M[col][j];
      v[r] -= f * v[col];
    }
  }
  for (int i = 0; i < np; ++i) a[i] = v[i] / M[i][i];
  *sigma0 = a[0];
  *delta = -a[1] / (2.0 * a[0]);
  *cc = quadratic ? a[2] / a[0] : 0.0;
  return LBM_OK;
}

// ---------------------------------------------------------------- z-slab decomposition
// One lattice split along z over several processes.  The update of Eq. (3) is
// local (Sec. II, below Eq. (3)): a node's new populations depend on the stored
// populations of the nodes within R + 1 planes (pull, then the density of the
// psi neighbours within R).  Each slab is stepped as a periodic lattice of its
// owned planes plus R + 1 ghost planes on each side; wrap-around then reaches
// only ghost planes, and after every step the ghost planes' needed populations
// are copied from the neighbouring slabs.

lbm_status lbm_slab_partition(int nz, int world, int stencil, int* z_begin) {
  if (!z_begin) return fail(nullptr, LBM_EINVAL, "z_begin is null");
  if (!valid_stencil(stencil)) return fail(nullptr, LBM_EINVAL, "stencil must be 4, 6 or 8");
  if (world < 1 || nz < 1) return fail(nullptr, LBM_EINVAL, "nz and world must be >= 1");
  const int H = radius_of(stencil) + 1;
  if (nz / world < H)
    return fail(nullptr, LBM_EINVAL, "%d planes over %d slabs leave fewer than %d planes in a slab", nz, world, H);
  const int base = nz / world, extra = nz % world;
  z_begin[0] = 0;
  for (int r = 0; r < world; ++r) z_begin[r + 1] = z_begin[r] + base + (r < extra ? 1 : 0);
  return LBM_OK;
}

lbm_status lbm_slab_halo_mask(int stencil, int side, int k, unsigned* mask) {
  if (!mask) return fail(nullptr, LBM_EINVAL, "mask is null");
  if (!valid_stencil(stencil)) return fail(nullptr, LBM_EINVAL, "stencil must be 4, 6 or 8");
  const int R = radius_of(stencil);
  if ((side != -1 && side != 1) || k < 1 || k > R + 1)
    return fail(nullptr, LBM_EINVAL, "side must be -1 or +1 and k in 1..%d", R + 1);
  // Stored slot i of node y streams to y + xi_i.  Ghost plane k below the slab
  // (z0 - k) feeds the pull of owned plane z0 (k = 1, c_z = +1) and the density
  // of ghost planes z0 - j, j = 1..R, which pulls slot i from plane z0 - j - c_z:
  // c_z = +1 is needed for k <= R + 1, c_z = 0 for k <= R, c_z = -1 for
  // k <= R - 1.  Above the slab the signs of c_z swap.
  unsigned m = 0;
  for (int i = 0; i < Q; ++i) {
    const int c = side * cz(i);   // +1: towards the slab
    const bool need = c == -1 ? k <= R + 1 : (c == 0 ? k <= R : k <= R - 1);
    if (need) m |= 1u << i;
  }
  *mask = m;
  return LBM_OK;
}

lbm_status lbm_set_populations_storage(lbm_ctx* c, const double* host_f, double n0, double scale) {
  LBM_CHECK_CTX(c);
  if (!(isfinite(n0) && isfinite(scale) && scale > 0))
    return fail(c, LBM_EINVAL, "n0 must be finite and scale positive");
  if (c->prec != kF16 && scale != 1.0) return fail(c, LBM_EINVAL, "scale must be 1 for FP64 and FP32 storage");
  int ex = 0;
  if (c->prec == kF16 && frexp(scale, &ex) != 0.5) return fail(c, LBM_EINVAL, "scale must be a power of two");
  lbm_status st = lbm_set_populations(c, host_f);
  if (st != LBM_OK || c->prec == kF64) return st;
  // rewrite the field under the given storage parameters
  c->n0 = n0;
  c->scale = scale;
  const long long N = (long long)c->box.nx * c->box.ny * c->box.nz;
  double* tmp = static_cast<double*>(c->pop[1]);
  LatticeDesc d = desc_of(c, 1);   // writes pop[0]
  for (int i = 0; i < Q; ++i) {
    LBM_CUDA(c, cudaMemcpyAsync(tmp, host_f + (long long)i * N, N * sizeof(double),
                                cudaMemcpyHostToDevice, c->stream));
    LBM_CUDA(c, launch_set_plane(c->prec, d, i, tmp, c->stream));
  }
  return reset_history(c);
}

lbm_status lbm_state_plane(const lbm_ctx* c, int i, int z, void** dev_ptr, size_t* bytes) {
  if (!c) return fail(nullptr, LBM_EINVAL, "null context");
  if (!dev_ptr || !bytes) return fail(nullptr, LBM_EINVAL, "dev_ptr or bytes is null");
  if (i < 0 || i >= Q || z < 0 || z >= c->box.nz) return fail(nullptr, LBM_EINVAL, "population or plane out of range");
  const size_t es = c->prec == kF64 ? 8 : (c->prec == kF32 ? 4 : 2);
  const size_t plane = (size_t)c->box.nx * c->box.ny;
  *bytes = plane * es;
  *dev_ptr = static_cast<char*>(c->pop[c->cur]) + ((size_t)i * c->box.nz + z) * plane * es;
  return LBM_OK;
}

lbm_status lbm_halo_copy(lbm_ctx* dst, int dst_z, const lbm_ctx* src, int src_z, unsigned mask) {
  LBM_CHECK_CTX(dst);
  if (!src) return fail(dst, LBM_EINVAL, "src is null");
  if (src->box.nx != dst->box.nx || src->box.ny != dst->box.ny || src->prec != dst->prec ||
      src->n0 != dst->n0 || src->scale != dst->scale)
    return fail(dst, LBM_EINVAL, "slabs differ in plane size, storage precision or storage parameters");
  if (mask >> Q) return fail(dst, LBM_EINVAL, "mask has bits above population %d", Q - 1);
  if (dst_z < 0 || dst_z >= dst->box.nz || src_z < 0 || src_z >= src->box.nz)
    return fail(dst, LBM_EINVAL, "plane out of range");
  if (src != dst && src->stream != dst->stream) {
    // the copy follows the source's queued steps
    cudaEvent_t ev;
    LBM_CUDA(dst, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    cudaError_t e = cudaEventRecord(ev, src->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(dst->stream, ev, 0);
    cudaEventDestroy(ev);
    LBM_CUDA(dst, e);
  }
  for (int i = 0; i < Q; ++i) {
    if (!((mask >> i) & 1u)) continue;
    void *s = nullptr, *d = nullptr;
    size_t b = 0;
    lbm_state_plane(src, i, src_z, &s, &b);
    lbm_state_plane(dst, i, dst_z, &d, &b);
    LBM_CUDA(dst, cudaMemcpyAsync(d, s, b, cudaMemcpyDefault, dst->stream));
  }
  return LBM_OK;
}

}  // extern "C"

// ====================================================================== batches
//
// Many independent lattices (uneven boxes, each its own G, psi, tau) share one
// caller-owned workspace cut into equal slots.  Runs wait in a queue; a free
// slot takes the next run.  Every step advances all active lattices with one
// launch of the batch kernel (a table of lattices in device memory), captured
// in a CUDA graph of check_every launches; between graph launches the
// observables of every active lattice are measured (one synchronisation) and
// the converged ones free their slots.

#include "lbm_kernels_async.cuh"

namespace {

struct BatchRun {
  lbm_box box;
  double tau, G;
  lbm_eos eos;
  double center[3], R, rho_in, rho_out, width;
  int state = 0;            // 0 queued, 1 running, 2 finished
  lbm_status result = LBM_OK;
  lbm_obs obs{};
};

}  // namespace

struct lbm_batch {
  int slots;
  lbm_box max_box;
  int stencil, prec;
  cudaStream_t stream;
  cudaStream_t cap_stream;
  char* ws;
  size_t slot_bytes;
  BatchEntry* table_dev;
  BatchHeader* hdr_dev;
  std::vector<lbm_ctx*> slot_ctx;
  std::vector<int> slot_run;
  std::vector<BatchRun> runs;
  size_t next_queued = 0;
  std::vector<BatchEntry> table_host;
  BatchHeader hdr_host{};
  std::vector<lbm_obs> obs_host;
  cudaGraphExec_t graph = nullptr;
  int graph_len = 0;
  int graph_mode = -1;       // BatchMode the graph (and the table's tiling) was made for
  long long lattice_updates = 0;
  // configuration chosen by lbm_batch_autotune (defaults: the natural kernel mode,
  // z chunks of min(16, nz), every slot)
  int mode_override = -1;
  int zchunk = 0;
  int slot_cap = 0;
  std::vector<int> requeued;  // runs returned to the queue (started before next_queued)
  char err[512];
};

namespace {

lbm_status bfail(lbm_batch* b, lbm_status s, const char* fmt, ...) {
  char* buf = b ? b->err : g_err;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, 512, fmt, ap);
  va_end(ap);
  return s;
}

#define LBM_BCUDA(b, call)                                                               \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return bfail((b), LBM_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));      \
  } while (0)

struct BatchLayout {
  size_t slot, table, hdr, total;
};

BatchLayout batch_layout(int slots, lbm_box max_box, int stencil, int prec) {
  BatchLayout L;
  L.slot = lbm_workspace_bytes(max_box, stencil, prec);
  L.table = align256(sizeof(BatchEntry) * (size_t)slots);
  L.hdr = align256(sizeof(BatchHeader));
  L.total = L.slot * (size_t)slots + L.table + L.hdr;
  return L;
}

// kernel mode of the whole queue: the moment kernel needs tau = 1 and boxes whose
// rows split into 16-byte chunks (nx % 4 == 0) at least a tile plus apron wide
int natural_batch_mode(const lbm_batch* b);

// the kernel modes that can run the whole queue, fastest first by construction
std::vector<int> batch_modes_allowed(int natural, int prec) {
  if (prec == kF16) return {kBatchMoment};   // the only FP16 batch kernel
  if (natural == kBatchMoment) return {kBatchMoment, kBatchMomentElem, kBatchUnitTau};
  if (natural == kBatchMomentElem) return {kBatchMomentElem, kBatchUnitTau};
  return {natural};
}

int batch_mode(const lbm_batch* b) {
  const int natural = natural_batch_mode(b);
  if (b->mode_override >= 0)
    for (int m : batch_modes_allowed(natural, b->prec))
      if (m == b->mode_override) return m;
  return natural;
}

int natural_batch_mode(const lbm_batch* b) {
  bool unit = true, moment = true;
  const int bx = batch_tile(b->prec, b->stencil, kBatchMoment).bx;
  for (const BatchRun& r : b->runs) {
    if (r.tau != 1.0) unit = false;
    if (r.box.nx % 4 != 0 || r.box.nx < bx + 8) moment = false;
  }
  return !unit ? kBatchMixedTau : (moment ? kBatchMoment : kBatchMomentElem);
}

lbm_status batch_fill(lbm_batch* b) {
  const int cap = b->slot_cap > 0 && b->slot_cap < b->slots ? b->slot_cap : b->slots;
  for (int k = 0; k < cap; ++k) {
    while (!b->slot_ctx[k] && (!b->requeued.empty() || b->next_queued < b->runs.size())) {
      int id;
      if (!b->requeued.empty()) {
        id = b->requeued.back();
        b->requeued.pop_back();
      } else {
        id = (int)b->next_queued++;
      }
      BatchRun& r = b->runs[id];
      lbm_ctx* c = nullptr;
      lbm_status st = lbm_create(r.box, r.tau, r.G, r.eos, b->stencil, b->prec, b->ws + k * b->slot_bytes,
                                 b->slot_bytes, b->stream, &c);
      if (st == LBM_OK) st = lbm_init_drop(c, r.center, r.R, r.rho_in, r.rho_out, r.width);
      if (st == LBM_OK) st = lbm_observables(c, &r.obs);   // reference Delta P and velocity
      if (st != LBM_OK) {
        r.state = 2;
        r.result = st;
        if (c) {
          snprintf(b->err, sizeof(b->err), "run %d: %s", id, c->err);
          lbm_destroy(c);
        } else {
          snprintf(b->err, sizeof(b->err), "run %d: %s", id, g_err);
        }
        if (st == LBM_ECUDA) return st;
        continue;
      }
      r.state = 1;
      b->slot_ctx[k] = c;
      b->slot_run[k] = id;
    }
  }
  return LBM_OK;
}

// table of the active lattices, in slot order, with their global work items
lbm_status batch_upload(lbm_batch* b) {
  const TileCfg t = batch_tile(b->prec, b->stencil, b->graph_mode);
  b->table_host.clear();
  long long items = 0;
  for (int k = 0; k < b->slots; ++k) {
    lbm_ctx* c = b->slot_ctx[k];
    if (!c) continue;
    BatchEntry e;
    e.d = desc_of(c, 0);
    e.parity = c->cur;
    const int zc = b->zchunk > 0 ? b->zchunk : 16;
    e.zchunk = c->box.nz < zc ? c->box.nz : zc;
    e.item_begin = items;
    items += (long long)((c->box.nx + t.bx - 1) / t.bx) * ((c->box.ny + t.by - 1) / t.by) *
             ((c->box.nz + e.zchunk - 1) / e.zchunk);
    b->table_host.push_back(e);
  }
  b->hdr_host.n = (int)b->table_host.size();
  b->hdr_host.total_items = items;
  if (!b->table_host.empty())
    LBM_BCUDA(b, cudaMemcpyAsync(b->table_dev, b->table_host.data(),
                                      sizeof(BatchEntry) * b->table_host.size(), cudaMemcpyHostToDevice,
                                      b->stream));
  LBM_BCUDA(b, cudaMemcpyAsync(b->hdr_dev, &b->hdr_host, sizeof(BatchHeader), cudaMemcpyHostToDevice,
                                    b->stream));
  LBM_BCUDA(b, cudaStreamSynchronize(b->stream));   // host copies of the table are reused
  return LBM_OK;
}

lbm_status batch_graph(lbm_batch* b, int len, int mode) {
  if (b->graph && b->graph_len == len && b->graph_mode == mode) return LBM_OK;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  int grid = 0;
  LBM_BCUDA(b, launch_batch(b->prec, b->stencil, mode, b->table_dev, b->hdr_dev, 0, true, &grid,
                                 b->stream));
  cudaGraph_t g = nullptr;
  LBM_BCUDA(b, cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < len && e == cudaSuccess; ++k)
    e = launch_batch(b->prec, b->stencil, mode, b->table_dev, b->hdr_dev, k & 1, false, nullptr,
                     b->cap_stream);
  cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &g);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return bfail(b, LBM_ECUDA, "batch graph capture failed: %s",
                 cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  e = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    b->graph = nullptr;
    return bfail(b, LBM_ECUDA, "batch graph instantiate failed: %s", cudaGetErrorString(e));
  }
  b->graph_len = len;
  b->graph_mode = mode;
  return LBM_OK;
}

void batch_finish(lbm_batch* b, int k, lbm_status result, int criterion) {
  BatchRun& r = b->runs[b->slot_run[k]];
  r.obs = b->slot_ctx[k]->last;
  r.obs.criterion = criterion;
  r.result = result;
  r.state = 2;
  lbm_destroy(b->slot_ctx[k]);
  b->slot_ctx[k] = nullptr;
  b->slot_run[k] = -1;
}

}  // namespace

extern "C" {

size_t lbm_batch_workspace_bytes(int slots, lbm_box max_box, int stencil, int prec) {
  if (slots < 1 || lbm_workspace_bytes(max_box, stencil, prec) == 0) return 0;
  if (prec == kF16 && stencil != 4) return 0;   // FP16 batches: the E4 moment kernel only
  return batch_layout(slots, max_box, stencil, prec).total;
}

lbm_status lbm_batch_create(int slots, lbm_box max_box, int stencil, int prec, void* dev_workspace,
                            size_t bytes, void* cuda_stream, lbm_batch** out) {
  if (!out) return bfail(nullptr, LBM_EINVAL, "out is null");
  *out = nullptr;
  if (slots < 1) return bfail(nullptr, LBM_EINVAL, "slots must be >= 1");
  if (!valid_stencil(stencil) || !valid_prec(prec) || (prec == kF16 && stencil != 4))
    return bfail(nullptr, LBM_EINVAL, "batches need stencil 4/6/8 (4 for F16 storage)");
  if (!box_ok(max_box, stencil)) return bfail(nullptr, LBM_EINVAL, "max_box not allowed (sides >= 2R + 1, below 2^31 nodes)");
  const BatchLayout L = batch_layout(slots, max_box, stencil, prec);
  if (!dev_workspace) return bfail(nullptr, LBM_EINVAL, "workspace is null");
  if (((uintptr_t)dev_workspace & 255) != 0) return bfail(nullptr, LBM_EINVAL, "workspace not 256-byte aligned");
  if (bytes < L.total) return bfail(nullptr, LBM_ENOMEM, "workspace has %zu bytes, needs %zu", bytes, L.total);
  lbm_batch* b = new lbm_batch();
  b->err[0] = 0;
  b->slots = slots;
  b->max_box = max_box;
  b->stencil = stencil;
  b->prec = prec;
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  b->ws = static_cast<char*>(dev_workspace);
  b->slot_bytes = L.slot;
  b->table_dev = reinterpret_cast<BatchEntry*>(b->ws + L.slot * (size_t)slots);
  b->hdr_dev = reinterpret_cast<BatchHeader*>(b->ws + L.slot * (size_t)slots + L.table);
  b->slot_ctx.assign(slots, nullptr);
  b->slot_run.assign(slots, -1);
  cudaError_t e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete b;
    return bfail(nullptr, LBM_ECUDA, "cudaStreamCreate failed: %s", cudaGetErrorString(e));
  }
  *out = b;
  return LBM_OK;
}

void lbm_batch_destroy(lbm_batch* b) {
  if (!b) return;
  for (lbm_ctx* c : b->slot_ctx)
    if (c) lbm_destroy(c);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  delete b;
}

lbm_status lbm_batch_enqueue(lbm_batch* b, lbm_box box, double tau, double G, lbm_eos eos,
                             const double center[3], double R, double rho_in, double rho_out,
                             double width, int* id) {
  if (!b) return bfail(nullptr, LBM_EINVAL, "null batch");
  if (!center || !id) return bfail(b, LBM_EINVAL, "center and id must not be null");
  if (box.nx > b->max_box.nx || box.ny > b->max_box.ny || box.nz > b->max_box.nz || !box_ok(box, b->stencil))
    return bfail(b, LBM_EINVAL, "box %dx%dx%d does not fit the batch's slots", box.nx, box.ny, box.nz);
  if (b->prec == kF16 && (tau != 1.0 || box.nx % 8 != 0 || box.nx < 48))
    return bfail(b, LBM_EINVAL, "F16 batches take tau = 1 and nx %% 8 == 0, nx >= 48 (the FP16 moment kernel)");
  BatchRun r;
  r.box = box;
  r.tau = tau;
  r.G = G;
  r.eos = eos;
  for (int k = 0; k < 3; ++k) r.center[k] = center[k];
  r.R = R;
  r.rho_in = rho_in;
  r.rho_out = rho_out;
  r.width = width;
  b->runs.push_back(r);
  *id = (int)b->runs.size() - 1;
  return LBM_OK;
}

lbm_status lbm_batch_run(lbm_batch* b, long long max_steps, long long check_every, double tol_dP_rel,
                         double tol_du, long long* lattice_updates) {
  NvtxRange nvtx("lbm_batch_run");
  if (!b) return bfail(nullptr, LBM_EINVAL, "null batch");
  if (max_steps < 0 || check_every < 2) return bfail(b, LBM_EINVAL, "max_steps >= 0, check_every >= 2");
  const int K = (int)(check_every + (check_every & 1));   // even: a graph keeps every parity
  const int mode = batch_mode(b);
  lbm_status st = batch_fill(b);
  if (st != LBM_OK) return st;
  st = batch_graph(b, K, mode);
  if (st != LBM_OK) return st;
  for (;;) {
    int active = 0;
    for (lbm_ctx* c : b->slot_ctx) active += c != nullptr;
    if (!active) break;
    st = batch_upload(b);
    if (st != LBM_OK) return st;
    LBM_BCUDA(b, cudaGraphLaunch(b->graph, b->stream));
    b->obs_host.assign(b->slots, lbm_obs{});
    for (int k = 0; k < b->slots; ++k) {
      lbm_ctx* c = b->slot_ctx[k];
      if (!c) continue;
      c->steps += K;
      b->lattice_updates += (long long)K * c->box.nx * c->box.ny * c->box.nz;
      st = observe(c, nullptr, nullptr, 1, true);
      if (st != LBM_OK) return bfail(b, st, "%s", c->err);
      LBM_BCUDA(b, cudaMemcpyAsync(&b->obs_host[k], c->obs_dev, sizeof(lbm_obs), cudaMemcpyDeviceToHost,
                                        b->stream));
    }
    LBM_BCUDA(b, cudaStreamSynchronize(b->stream));
    for (int k = 0; k < b->slots; ++k) {
      lbm_ctx* c = b->slot_ctx[k];
      if (!c) continue;
      const unsigned prev_bits = c->last.status_bits;
      c->last = b->obs_host[k];
      c->have_u_old = 1;
      c->have_last = 1;
      if (c->last.status_bits & 16u) batch_finish(b, k, LBM_ETIMEOUT, 0);
      else if (c->last.status_bits & 8u) batch_finish(b, k, LBM_ENUMERIC, 0);
      // collapsed at two checks in a row: the droplet/bubble is gone for good and the
      // run can no longer give a point of the sweep; its slot is freed
      else if ((c->last.status_bits & 2u) && (prev_bits & 2u)) batch_finish(b, k, LBM_ECOLLAPSE, 0);
      else if (c->last.dP_rel_change < tol_dP_rel) batch_finish(b, k, LBM_OK, 1);
      else if (c->last.du < tol_du) batch_finish(b, k, LBM_OK, 2);
      else if (c->steps >= max_steps) batch_finish(b, k, LBM_ENOTCONV, 0);
    }
    st = batch_fill(b);
    if (st != LBM_OK) return st;
  }
  if (lattice_updates) *lattice_updates = b->lattice_updates;
  return LBM_OK;
}

lbm_status lbm_batch_autotune(lbm_batch* b, int reps, long long* choice) {
  NvtxRange nvtx("lbm_batch_autotune");
  if (!b) return bfail(nullptr, LBM_EINVAL, "null batch");
  if (reps < 2) reps = 2;
  reps += reps & 1;
  lbm_status st = batch_fill(b);
  if (st != LBM_OK) return st;
  std::vector<int> filled;
  for (int k = 0; k < b->slots; ++k)
    if (b->slot_ctx[k]) filled.push_back(k);
  if (filled.empty()) return bfail(b, LBM_EINVAL, "autotune needs queued runs");
  const int natural = natural_batch_mode(b);
  std::vector<int> caps = {b->slots};
  if ((int)filled.size() >= 4) caps.push_back((b->slots + 1) / 2);
  cudaEvent_t e0, e1;
  LBM_BCUDA(b, cudaEventCreate(&e0));
  LBM_BCUDA(b, cudaEventCreate(&e1));
  int best_mode = natural, best_zc = 0, best_cap = b->slots;
  double best_rate = -1.0;
  const int save_cap = b->slot_cap;
  for (int mode : batch_modes_allowed(natural, b->prec)) {
    for (int zc : {8, 16, 32}) {
      for (int cap : caps) {
        b->mode_override = mode;
        b->zchunk = zc;
        b->slot_cap = cap;   // the first `cap` slots take part in the measurement
        long long nodes = 0;
        for (int k = 0; k < b->slots && k < cap; ++k)
          if (b->slot_ctx[k]) nodes += (long long)b->slot_ctx[k]->box.nx * b->slot_ctx[k]->box.ny * b->slot_ctx[k]->box.nz;
        if (!nodes) continue;
        // time `reps` launches over the table restricted to the first cap slots
        std::vector<lbm_ctx*> hidden(b->slots, nullptr);
        for (int k = cap; k < b->slots; ++k) std::swap(hidden[k], b->slot_ctx[k]);
        b->graph_mode = mode;   // the table's tiling follows the kernel launched
        st = batch_upload(b);
        int grid = 0;
        cudaError_t ce = cudaSuccess;
        if (st == LBM_OK)
          ce = launch_batch(b->prec, b->stencil, mode, b->table_dev, b->hdr_dev, 0, true, &grid, b->stream);
        for (int r = 0; r < 2 && st == LBM_OK && ce == cudaSuccess; ++r)
          ce = launch_batch(b->prec, b->stencil, mode, b->table_dev, b->hdr_dev, r & 1, false, nullptr, b->stream);
        if (st == LBM_OK && ce == cudaSuccess) ce = cudaEventRecord(e0, b->stream);
        for (int r = 0; r < reps && st == LBM_OK && ce == cudaSuccess; ++r)
          ce = launch_batch(b->prec, b->stencil, mode, b->table_dev, b->hdr_dev, r & 1, false, nullptr, b->stream);
        if (st == LBM_OK && ce == cudaSuccess) ce = cudaEventRecord(e1, b->stream);
        if (st == LBM_OK && ce == cudaSuccess) ce = cudaEventSynchronize(e1);
        for (int k = cap; k < b->slots; ++k) std::swap(hidden[k], b->slot_ctx[k]);
        if (st != LBM_OK || ce != cudaSuccess) {
          cudaEventDestroy(e0);
          cudaEventDestroy(e1);
          b->slot_cap = save_cap;
          b->mode_override = -1;
          b->zchunk = 0;
          return st != LBM_OK ? st : bfail(b, LBM_ECUDA, "batch autotune: %s", cudaGetErrorString(ce));
        }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        const double rate = (double)nodes * reps / (ms * 1e-3);
        if (rate > best_rate) {
          best_rate = rate;
          best_mode = mode;
          best_zc = zc;
          best_cap = cap;
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->mode_override = best_mode;
  b->zchunk = best_zc;
  b->slot_cap = best_cap;
  // the timed launches advanced the resident lattices: start them again from their
  // initial drops; those beyond the chosen slot count go back to the queue
  for (int k = 0; k < b->slots; ++k) {
    lbm_ctx* c = b->slot_ctx[k];
    if (!c) continue;
    const int id = b->slot_run[k];
    BatchRun& r = b->runs[id];
    if (k >= best_cap) {
      lbm_destroy(c);
      b->slot_ctx[k] = nullptr;
      b->slot_run[k] = -1;
      r.state = 0;
      b->requeued.push_back(id);
      continue;
    }
    st = lbm_init_drop(c, r.center, r.R, r.rho_in, r.rho_out, r.width);
    if (st == LBM_OK) st = lbm_observables(c, &r.obs);
    if (st != LBM_OK) return bfail(b, st, "run %d: %s", id, c->err);
  }
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  b->graph_mode = -1;
  if (choice) *choice = (long long)best_mode * 1000000 + (long long)best_zc * 1000 + best_cap;
  return LBM_OK;
}

lbm_status lbm_batch_result(const lbm_batch* b, int id, lbm_obs* out) {
  if (!b || !out) return bfail(nullptr, LBM_EINVAL, "null argument");
  if (id < 0 || id >= (int)b->runs.size()) return bfail(nullptr, LBM_EINVAL, "no run %d", id);
  const BatchRun& r = b->runs[id];
  if (r.state != 2) return bfail(nullptr, LBM_EINVAL, "run %d has not finished", id);
  *out = r.obs;
  return r.result;
}

const char* lbm_batch_last_error(const lbm_batch* b) { return b ? b->err : g_err; }

}  // extern "C"

// ---------------------------------------------------------------- groups of lattices

struct lbm_group {
  std::vector<lbm_ctx*> ctx;
  int stencil, prec, mode;
  cudaStream_t stream;
  cudaStream_t cap_stream;
  BatchEntry* table_dev;
  BatchHeader* hdr_dev;
  std::vector<BatchEntry> table_host;
  BatchHeader hdr_host{};
  int grid = 0;
  cudaGraphExec_t graph = nullptr;
  int graph_len = 128;        // even: a replay keeps every lattice's parity
  char err[512];
};

namespace {

lbm_status gfail(lbm_group* g, lbm_status s, const char* fmt, ...) {
  char* buf = g ? g->err : g_err;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, 512, fmt, ap);
  va_end(ap);
  return s;
}

#define LBM_GCUDA(g, call)                                                               \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return gfail((g), LBM_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));      \
  } while (0)

// the table of the group's lattices with their current parities; one z chunk for
// all of them, chosen like the single-lattice launcher (fewest rounds x planes)
lbm_status group_upload(lbm_group* g) {
  const TileCfg t = batch_tile(g->prec, g->stencil, g->mode);
  const int R = radius_of(g->stencil);
  int max_nz = 1;
  for (lbm_ctx* c : g->ctx) max_nz = c->box.nz > max_nz ? c->box.nz : max_nz;
  int best_zc = max_nz;
  long long best_cost = -1;
  for (int zc = 1; zc <= max_nz; ++zc) {
    long long items = 0;
    for (lbm_ctx* c : g->ctx)
      items += (long long)((c->box.nx + t.bx - 1) / t.bx) * ((c->box.ny + t.by - 1) / t.by) *
               ((c->box.nz + zc - 1) / zc);
    const long long rounds = (items + g->grid - 1) / g->grid;
    const long long cost = rounds * (zc + 2 * R);
    if (best_cost < 0 || cost <= best_cost) {
      best_cost = cost;
      best_zc = zc;
    }
  }
  g->table_host.clear();
  long long items = 0;
  for (lbm_ctx* c : g->ctx) {
    BatchEntry e;
    e.d = desc_of(c, 0);
    e.parity = c->cur;
    e.zchunk = best_zc < c->box.nz ? best_zc : c->box.nz;
    e.item_begin = items;
    items += (long long)((c->box.nx + t.bx - 1) / t.bx) * ((c->box.ny + t.by - 1) / t.by) *
             ((c->box.nz + e.zchunk - 1) / e.zchunk);
    g->table_host.push_back(e);
  }
  g->hdr_host.n = (int)g->table_host.size();
  g->hdr_host.total_items = items;
  LBM_GCUDA(g, cudaMemcpyAsync(g->table_dev, g->table_host.data(), sizeof(BatchEntry) * g->table_host.size(),
                               cudaMemcpyHostToDevice, g->stream));
  LBM_GCUDA(g, cudaMemcpyAsync(g->hdr_dev, &g->hdr_host, sizeof(BatchHeader), cudaMemcpyHostToDevice, g->stream));
  LBM_GCUDA(g, cudaStreamSynchronize(g->stream));   // the host copy is reused
  return LBM_OK;
}

}  // namespace

size_t lbm_group_workspace_bytes(int n) {
  if (n < 1) return 0;
  return align256(sizeof(BatchEntry) * (size_t)n) + align256(sizeof(BatchHeader));
}

lbm_status lbm_group_create(lbm_ctx* const* ctxs, int n, void* dev_workspace, size_t bytes,
                            void* cuda_stream, lbm_group** out) {
  if (!out) return gfail(nullptr, LBM_EINVAL, "out is null");
  *out = nullptr;
  if (!ctxs || n < 1) return gfail(nullptr, LBM_EINVAL, "need n >= 1 contexts");
  if (!dev_workspace || ((uintptr_t)dev_workspace & 255) != 0)
    return gfail(nullptr, LBM_EINVAL, "workspace null or not 256-byte aligned");
  if (bytes < lbm_group_workspace_bytes(n))
    return gfail(nullptr, LBM_ENOMEM, "workspace has %zu bytes, needs %zu", bytes, lbm_group_workspace_bytes(n));
  for (int k = 0; k < n; ++k) {
    if (!ctxs[k]) return gfail(nullptr, LBM_EINVAL, "context %d is null", k);
    for (int j = 0; j < k; ++j)
      if (ctxs[j] == ctxs[k]) return gfail(nullptr, LBM_EINVAL, "context %d appears twice", k);
    if (ctxs[k]->prec != ctxs[0]->prec || ctxs[k]->stencil != ctxs[0]->stencil)
      return gfail(nullptr, LBM_EINVAL, "all contexts need the same storage and stencil");
  }
  if (ctxs[0]->prec == kF16) return gfail(nullptr, LBM_EINVAL, "groups need F64 or F32 storage");
  lbm_group* g = new lbm_group();
  g->err[0] = 0;
  g->ctx.assign(ctxs, ctxs + n);
  g->stencil = ctxs[0]->stencil;
  g->prec = ctxs[0]->prec;
  g->stream = static_cast<cudaStream_t>(cuda_stream);
  char* ws = static_cast<char*>(dev_workspace);
  g->table_dev = reinterpret_cast<BatchEntry*>(ws);
  g->hdr_dev = reinterpret_cast<BatchHeader*>(ws + align256(sizeof(BatchEntry) * (size_t)n));
  // kernel mode as for a batch: the moment kernel when every lattice allows it
  bool unit = true, moment = true;
  const int bx = batch_tile(g->prec, g->stencil, kBatchMoment).bx;
  for (lbm_ctx* c : g->ctx) {
    if (c->tau != 1.0) unit = false;
    if (c->box.nx % 4 != 0 || c->box.nx < bx + 8) moment = false;
  }
  g->mode = !unit ? kBatchMixedTau : (moment ? kBatchMoment : kBatchMomentElem);
  cudaError_t e = cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess)
    e = launch_batch(g->prec, g->stencil, g->mode, g->table_dev, g->hdr_dev, 0, true, &g->grid, g->stream);
  if (e != cudaSuccess) {
    if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
    delete g;
    return gfail(nullptr, LBM_ECUDA, "group set-up failed: %s", cudaGetErrorString(e));
  }
  *out = g;
  return LBM_OK;
}

void lbm_group_destroy(lbm_group* g) {
  if (!g) return;
  if (g->graph) cudaGraphExecDestroy(g->graph);
  if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
  delete g;
}

lbm_status lbm_group_step(lbm_group* g, long long n) {
  NvtxRange nvtx("lbm_group_step");
  if (!g) return gfail(nullptr, LBM_EINVAL, "null group");
  if (n < 0) return gfail(g, LBM_EINVAL, "n must be >= 0");
  for (lbm_ctx* c : g->ctx)
    if (!c->initialised) return gfail(g, LBM_EINVAL, "a lattice of the group is not initialised");
  if (n == 0) return LBM_OK;
  // the table holds each lattice's buffer parity: write it again (and drop the
  // graph captured with the old table) when any lattice's parity has changed, e.g.
  // after an odd number of steps or a lattice stepped on its own
  bool stale = g->table_host.size() != g->ctx.size();
  for (size_t k = 0; !stale && k < g->ctx.size(); ++k) stale = g->table_host[k].parity != g->ctx[k]->cur;
  if (stale) {
    lbm_status st = group_upload(g);
    if (st != LBM_OK) return st;
    if (g->graph) cudaGraphExecDestroy(g->graph);
    g->graph = nullptr;
  }
  if (n >= g->graph_len && !g->graph) {
    cudaGraph_t gr = nullptr;
    LBM_GCUDA(g, cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < g->graph_len && e == cudaSuccess; ++k)
      e = launch_batch(g->prec, g->stencil, g->mode, g->table_dev, g->hdr_dev, k & 1, false, nullptr,
                       g->cap_stream);
    cudaError_t e2 = cudaStreamEndCapture(g->cap_stream, &gr);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (gr) cudaGraphDestroy(gr);
      return gfail(g, LBM_ECUDA, "group graph capture failed: %s",
                   cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(&g->graph, gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) {
      g->graph = nullptr;
      return gfail(g, LBM_ECUDA, "group graph instantiate failed: %s", cudaGetErrorString(e));
    }
  }
  long long done = 0;
  while (n - done >= g->graph_len) {
    LBM_GCUDA(g, cudaGraphLaunch(g->graph, g->stream));
    done += g->graph_len;
  }
  for (long long k = 0; done + k < n; ++k)
    LBM_GCUDA(g, launch_batch(g->prec, g->stencil, g->mode, g->table_dev, g->hdr_dev, (int)(k & 1), false,
                              nullptr, g->stream));
  for (lbm_ctx* c : g->ctx) {
    c->steps += n;
    c->cur ^= (int)(n & 1);
  }
  return LBM_OK;
}

const char* lbm_group_last_error(const lbm_group* g) { return g ? g->err : g_err; }

// ---------------------------------------------------------------- TMA tensor maps

bool lbm::build_tma_maps(TmaMaps* t, const void* pop0, const void* pop1, int nx, int ny, int nz, int R,
                         int bx, int by) {
  t->ok = 0;
  EncodeTiledFn enc = tensor_map_encoder();
  if (!enc || !tma_box_ok(nx, ny, nz, by) || R < 1 || R + 3 > kMaxTmaMaps) return false;
  const int XW = bx + 8, PY = by + 2 * R;   // the kernel's boxes (TmaShape)
  const cuuint64_t N = (cuuint64_t)nx * ny * nz;
  const cuuint64_t dims[4] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz, (cuuint64_t)Q};
  const cuuint64_t strides[3] = {(cuuint64_t)nx * 4, (cuuint64_t)nx * ny * 4, N * 4};
  const cuuint32_t es[4] = {1, 1, 1, 1};
  const void* base[2] = {pop0, pop1};
  for (int b = 0; b < 2; ++b) {
    if (((uintptr_t)base[b] & 15) != 0) return false;
    for (int k = 0; k <= R + 2; ++k) {
      // k = 0: the stage box; 1 .. R + 1: k wrapped rows; R + 2: the 16-byte x apron
      const cuuint32_t box[4] = {(cuuint32_t)(k == R + 2 ? 4 : XW), (cuuint32_t)(k == 0 || k == R + 2 ? PY : k), 1,
                                 1};
      const CUresult r = enc(&t->map[b][k], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void*>(base[b]), dims,
                             strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return false;
    }
    t->base[b] = base[b];
  }
  t->bx = bx;
  t->by = by;
  t->ok = 1;
  return true;
}
