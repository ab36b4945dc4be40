// C ABI of the solver: context, multigrid hierarchy, set-up calls and the
// FP64 / mixed-precision step drivers.  Each stage of a step is one of the
// kernels in k64.cu / k32.cu; the host only sequences launches and reads the
// 8-byte residual norms that drive the stop tests.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <thread>
#include <type_traits>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "launch.h"
#include "richards.h"
#include "validate.h"

using rich::Level;
using rich::Phys;
using rich::Xfer;
using rich::law_error;

namespace {

constexpr int MAXLEV = 24;
constexpr int NSCRATCH = 72;   // norm slots + statistics (32..63: the single-block step's; 64..66: the
                               // cooperative cycle's reductions; 67..71: the inner-loop graph's control)
// Levels of at most this many cells run as one cooperative launch: 0, off by
// default -- on the 256^3 drainage its grid barriers cost more than the
// graph-replayed stage launches they replace (32.8 ms per step without, 33.7
// with 16^3 and below, 35.0 with 64^3 and below); richards_set_coop turns it on
constexpr long long COOP_CELLS = 0;
constexpr int MASS_PARTS = 152 * 32;   // water-balance blocks (grid_for's cap)

struct HLevel {
  int n[3] = {1, 1, 1};
  double h[3] = {1, 1, 1};
  long long ncell = 0;
  long long nface[6] = {0, 0, 0, 0, 0, 0};
  double *u = nullptr, *ubar = nullptr, *g = nullptr, *d = nullptr, *Kc = nullptr;
  double *p1 = nullptr, *p2 = nullptr, *smax = nullptr;
  double* vgm = nullptr;         // finest level, van Genuchten n field: m = 1 - 1/n per cell
  double* kb[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  float *uf = nullptr, *ubarf = nullptr, *gf = nullptr, *df = nullptr, *Kcf = nullptr;
  float *p1f = nullptr, *p2f = nullptr, *smaxf = nullptr, *psi0f = nullptr;
  float* kbf[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  uint8_t* mat = nullptr;        // layered soil: material of each cell
  int cs = 0;                    // FP32 g, psi0, p1, p2, smax in the colour-split layout (rich::pix_of)
  // transfer tables to the next coarser level
  int *pc[3] = {}, *pj[3] = {}, *rc[3] = {}, *ri[3] = {};
  double *pw[3] = {}, *rw[3] = {};
  float *pwf[3] = {}, *rwf[3] = {};
};

// Progress of a context through its current step under a batcher, kept in
// the context between calls (a call can return with a context mid-step):
// which part of the step comes next, and the step's running values (those
// of step_mixed).
enum { BP_IDLE = 0, BP_DEFECT, BP_INNER, BP_FINISH };
struct BatchProgress {
  int phase = BP_IDLE;
  bool use64 = false;                  // FP64 outer layer: FP64 defects from here on
  bool predicted = false;
  double r = 0.0, r0 = 0.0, rin0 = 0.0, rtol_in = 0.0, r_ff = INFINITY;
  int outer = 0, inner = 0;            // outer iterations and inner cycles of the step
  int k = 0;                           // cycles of the current inner solve
  richards_status st = RICH_OK;        // RICH_ENOCONV once the outer limit is reached
  int nbal = 0;                        // water-balance partial sums in flight (finish)
  richards_status fin = RICH_OK;       // status of the finishing launches
};

}  // namespace

struct richards_ctx {
  cudaStream_t s = nullptr;
  richards_grid grid{};
  richards_opts opts{};
  int nlev = 0, tail_start = 0;
  HLevel L[MAXLEV];
  richards_soil soil{};
  bool soil_set = false, het_p1 = false, het_p2 = false, het_Ks = false;
  // layered soil (richards_set_materials): soil.model is then rich::COMPOSITE
  bool layered = false;
  int nmat = 0;
  richards_material mats[rich::MAXMAT] = {};
  rich::MatLaw<double>* dmat64 = nullptr;
  rich::MatLaw<float>* dmat32 = nullptr;
  rich::DDMat* dmatdd = nullptr;
  richards_bc bc{};
  bool bc_set = false;
  rich::BcDev bcdev{};
  richards_sink sink{};
  double *psi_n = nullptr, *psi_nm1 = nullptr, *Ks = nullptr;
  bool have_state = false, have_prev = false;
  // mixed mode: FP64 theta of psi^n, psi^{n-1} and of the latest iterate,
  // kept so that no step evaluates theta twice at the same state
  double *th_n = nullptr, *th_nm1 = nullptr, *th_cur = nullptr;
  bool th_n_valid = false, th_nm1_valid = false;
  double t = 0.0, a = 0.0, dt = 0.0;
  int scheme_used = 1;
  bool prepared = false;
  Level<double>* dL64 = nullptr;
  Xfer<double>* dX64 = nullptr;
  Level<float>* dL32 = nullptr;
  Xfer<float>* dX32 = nullptr;
  unsigned long long* scratch = nullptr;
  unsigned long long* hscratch = nullptr;    // pinned
  double* mass_part = nullptr;               // water-balance partial sums (+ the min bits)
  double* hmass = nullptr;                   // pinned
  std::vector<void*> allocs;
  std::vector<void*> bc_allocs;
  std::string err;
  long long updates_host = 0;
  // kernel timing (richards_profile)
  struct ProfRec { const char* name; int level; long long cells; cudaEvent_t a, b; };
  struct ProfAgg { long long launches = 0; double ms = 0.0; long long cells = 0; };
  int prof = 0;          // 0 off, 1 time every launch, 2 time level 0 and count the rest, 3 count only
  std::vector<ProfRec> prof_pending;
  std::vector<cudaEvent_t> ev_pool;
  std::map<std::pair<std::string, int>, ProfAgg> prof_agg;
  // richards_batch_submit: a worker thread runs the steps; the context is
  // busy (every other call returns EBUSY) until richards_batch_poll sees it done
  std::atomic<int> busy{0};
  std::thread worker;
  int device = 0;
  // CUDA graphs of the FP32 inner cycle, one per scheme (1: BDF1, 2: BDF2)
  struct GraphRec {
    cudaGraphExec_t exec = nullptr;
    double a = 0.0;
    int with_prof = 0;
    long long updates = 0;
    std::vector<ProfRec> prof;
  };
  GraphRec graphs[3];
  bool graphs_ok = true, capturing = false;
  // the whole FP32 inner solve as one graph (a conditional while node around
  // the cycle and its stop test), one per scheme; loop_ok: the device takes
  // conditional nodes
  struct LoopRec {
    cudaGraphExec_t exec = nullptr;
    double a = 0.0;
    long long updates = 0;             // NGS updates of one cycle
    std::vector<ProfRec> recs;         // the launches of one pass of the loop's body (counted, not timed)
  };
  LoopRec loops[3];
  bool loop_ok = true;
  std::string loop_err;
  std::string graph_status;             // richards_graph_status's message
  std::string graph_err;
  GraphRec* harvest = nullptr;
  std::vector<ProfRec> capture_recs;
  richards_status batch_status = RICH_OK;
  richards_step_info batch_info{};
  // launch shapes of the FP32 grid kernels per level (richards_autotune /
  // richards_set_launch; 0 = the defaults): cells per thread along z of the
  // half-sweeps, their block x-size, the defect kernel's block x-size
  int tune_planes[MAXLEV] = {}, tune_bx[MAXLEV] = {}, tune_rbx[MAXLEV] = {};
  // FP32 inner cycles: levels from coop_start down to the single-block tail
  // run as one cooperative launch (MAXLEV: none); its grid size
  int coop_start = MAXLEV, coop_blocks = 0;
  // batcher progress (richards_batcher_step / _advance); reset by any call
  // that prepares a step or changes the problem
  BatchProgress bp;
};

namespace {

richards_status fail(richards_ctx* c, richards_status st, const std::string& msg) {
  if (c) c->err = msg;
  return st;
}

#define CK(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) return fail(c, RICH_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <typename T>
richards_status dalloc(richards_ctx* c, T** p, long long n, std::vector<void*>* list = nullptr) {
  void* q = nullptr;
  size_t bytes = sizeof(T) * (size_t)(n > 0 ? n : 1);
  cudaError_t e = cudaMalloc(&q, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, RICH_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  (list ? list : &c->allocs)->push_back(q);
  *p = (T*)q;
  return RICH_OK;
}

#define TRY(x)                           \
  do {                                   \
    richards_status st_ = (x);           \
    if (st_ != RICH_OK) return st_;      \
  } while (0)

// ------------------------------------------------------------------------
// Kernel timing: CUDA events on the context's stream around each launch.
// ------------------------------------------------------------------------
cudaEvent_t prof_event(richards_ctx* c) {
  if (c->ev_pool.empty()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
  cudaEvent_t e = c->ev_pool.back();
  c->ev_pool.pop_back();
  return e;
}

void prof_count(richards_ctx* c, const char* name, int level, long long cells) {
  auto& g = c->prof_agg[{std::string(name), level}];
  g.launches += 1;
  g.cells += cells;
}

void prof_flush(richards_ctx* c) {
  if (c->prof_pending.empty()) return;
  cudaStreamSynchronize(c->s);
  for (auto& r : c->prof_pending) {
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    auto& g = c->prof_agg[{std::string(r.name), r.level}];
    g.launches += 1;
    g.ms += ms;
    g.cells += r.cells;
    c->ev_pool.push_back(r.a);
    c->ev_pool.push_back(r.b);
  }
  c->prof_pending.clear();
}

struct Prof {
  richards_ctx* c;
  const char* name;
  int level;
  long long cells;
  cudaEvent_t a = nullptr;
  // while a graph is captured the events become external event-record nodes,
  // so that their times can be read after each replay
  static void record(richards_ctx* c, cudaEvent_t e) {
    if (c->capturing) cudaEventRecordWithFlags(e, c->s, cudaEventRecordExternal);
    else cudaEventRecord(e, c->s);
  }
  Prof(richards_ctx* c_, const char* n, int l, long long cells_) : c(c_), name(n), level(l), cells(cells_) {
    if (c->prof == 1 || (c->prof == 2 && level == 0)) {
      a = prof_event(c);
      record(c, a);
    }
  }
  ~Prof() {
    if (!c->prof) return;
    if (!a) {                           // counted, not timed
      if (c->capturing) c->capture_recs.push_back({name, level, cells, nullptr, nullptr});
      else prof_count(c, name, level, cells);
      return;
    }
    cudaEvent_t b = prof_event(c);
    record(c, b);
    if (c->capturing) {                 // event nodes of a graph being captured
      c->capture_recs.push_back({name, level, cells, a, b});
      return;
    }
    c->prof_pending.push_back({name, level, cells, a, b});
    if (c->prof_pending.size() > 8192) prof_flush(c);
  }
};

// times of the event nodes of the graph replayed last (after a stream sync)
void graph_harvest(richards_ctx* c) {
  if (!c->harvest) return;
  for (auto& r : c->harvest->prof) {
    float ms = 0.0f;
    if (r.a) cudaEventElapsedTime(&ms, r.a, r.b);
    auto& g = c->prof_agg[{std::string(r.name), r.level}];
    g.launches += 1;
    g.ms += ms;
    g.cells += r.cells;
  }
  c->harvest = nullptr;
}

void graphs_reset(richards_ctx* c) {
  for (auto& g : c->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
    for (auto& r : g.prof)
      if (r.a) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    g.prof.clear();
  }
  for (auto& g : c->loops) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
  }
  c->harvest = nullptr;
}

bool finite_all(const double* a, long long n) {
  for (long long i = 0; i < n; ++i)
    if (!std::isfinite(a[i])) return false;
  return true;
}

// ------------------------------------------------------------------------
// Transfer tables along one axis.  Reading of "standard full weighting and
// linear interpolation" for cell-centred, possibly non-nested levels: the
// coarse coordinate of fine cell i is ((2i+1) nc - nf) / (2 nf); P mixes the
// two nearest coarse centres, folding a ghost beyond the end into the end
// cell with factor s (+1 constant extrapolation, -1 on a fully Dirichlet
// face); R is the transpose of P with s = +1, each row scaled to sum 1.
// ------------------------------------------------------------------------
struct Row {
  int cnt = 0;
  int idx[rich::RMAX];
  double w[rich::RMAX];
  bool add(int j, double wt) {
    if (wt == 0.0) return true;
    for (int k = 0; k < cnt; ++k)
      if (idx[k] == j) { w[k] += wt; return true; }
    if (cnt >= rich::RMAX) return false;
    idx[cnt] = j;
    w[cnt] = wt;
    ++cnt;
    return true;
  }
};

Row interp(int nf, int nc, int i, double slo, double shi) {
  Row r;
  if (nf == 1) { r.add(0, 1.0); return r; }
  const long long num = (long long)(2 * i + 1) * nc - nf, den = 2LL * nf;
  long long J0 = num >= 0 ? num / den : -((-num + den - 1) / den);
  const double w = (double)(num - J0 * den) / (double)den;
  const long long J1 = J0 + 1;
  if (J0 < 0) r.add(0, (1.0 - w) * slo); else r.add((int)J0, 1.0 - w);
  if (J1 >= nc) r.add(nc - 1, w * shi); else r.add((int)J1, w);
  return r;
}

// Rows of the restriction along one axis: the transpose of the
// constant-extrapolation interpolation, each row normalised to sum 1.
bool restriction_rows(int nf, int nc, std::vector<Row>& R) {
  R.assign(nc, Row());
  for (int i = 0; i < nf; ++i) {
    Row p0 = interp(nf, nc, i, 1.0, 1.0);
    for (int k = 0; k < p0.cnt; ++k)
      if (!R[p0.idx[k]].add(i, p0.w[k])) return false;
  }
  for (int J = 0; J < nc; ++J) {
    double s = 0.0;
    for (int k = 0; k < R[J].cnt; ++k) s += R[J].w[k];
    for (int k = 0; k < R[J].cnt; ++k) R[J].w[k] /= s;
  }
  return true;
}

richards_status build_axis_tables(richards_ctx* c, int l, int ax, double slo, double shi) {
  HLevel& F = c->L[l];
  HLevel& C = c->L[l + 1];
  const int nf = F.n[ax], nc = C.n[ax];
  std::vector<int> pc(nf), pj(2 * nf, 0), rc(nc, 0), ri((size_t)rich::RMAX * nc, 0);
  std::vector<double> pw(2 * nf, 0.0), rw((size_t)rich::RMAX * nc, 0.0);
  for (int i = 0; i < nf; ++i) {
    Row r = interp(nf, nc, i, slo, shi);
    pc[i] = r.cnt;
    for (int k = 0; k < r.cnt; ++k) { pj[2 * i + k] = r.idx[k]; pw[2 * i + k] = r.w[k]; }
  }
  std::vector<Row> R;
  if (!restriction_rows(nf, nc, R)) return fail(c, RICH_EINVAL, "restriction stencil too wide");
  for (int J = 0; J < nc; ++J) {
    rc[J] = R[J].cnt;
    for (int k = 0; k < R[J].cnt; ++k) {
      ri[rich::RMAX * J + k] = R[J].idx[k];
      rw[rich::RMAX * J + k] = R[J].w[k];
    }
  }
  std::vector<float> pwf(pw.begin(), pw.end()), rwf(rw.begin(), rw.end());
  auto up = [&](auto** dst, const auto& src) -> richards_status {
    using E = typename std::remove_reference<decltype(src)>::type::value_type;
    E* p;
    TRY(dalloc(c, &p, (long long)src.size(), &c->bc_allocs));
    CK(cudaMemcpy(p, src.data(), sizeof(E) * src.size(), cudaMemcpyHostToDevice));
    *dst = p;
    return RICH_OK;
  };
  TRY(up(&F.pc[ax], pc));
  TRY(up(&F.pj[ax], pj));
  TRY(up(&F.pw[ax], pw));
  TRY(up(&F.pwf[ax], pwf));
  TRY(up(&F.rc[ax], rc));
  TRY(up(&F.ri[ax], ri));
  TRY(up(&F.rw[ax], rw));
  TRY(up(&F.rwf[ax], rwf));
  return RICH_OK;
}

rich::Geom geom(const richards_ctx* c, int l) {
  rich::Geom G;
  G.dim = c->grid.dim;
  G.n0 = c->L[l].n[0];
  G.n1 = c->L[l].n[1];
  G.n2 = c->L[l].n[2];
  for (int a = 0; a < 3; ++a) G.h[a] = c->L[l].h[a];
  G.Lv = c->grid.L[c->grid.dim - 1];
  return G;
}

Level<double> view64(const richards_ctx* c, int l) {
  const HLevel& H = c->L[l];
  Level<double> V{};
  V.dim = c->grid.dim;
  V.n0 = H.n[0]; V.n1 = H.n[1]; V.n2 = H.n[2];
  V.ncell = H.ncell;
  for (int a = 0; a < 3; ++a) V.ih2[a] = a < c->grid.dim ? 1.0 / (H.h[a] * H.h[a]) : 0.0;
  V.u = H.u; V.ubar = H.ubar; V.g = H.g; V.d = H.d; V.Kc = H.Kc;
  V.p1 = c->het_p1 ? H.p1 : nullptr;
  V.p2 = c->het_p2 ? H.p2 : nullptr;
  V.smax = c->sink.enabled ? H.smax : nullptr;
  V.psi0 = nullptr;
  for (int f = 0; f < 6; ++f) V.kb[f] = H.kb[f];
  V.mat = c->layered ? H.mat : nullptr;
  return V;
}

Level<float> view32(const richards_ctx* c, int l) {
  const HLevel& H = c->L[l];
  Level<float> V{};
  V.dim = c->grid.dim;
  V.n0 = H.n[0]; V.n1 = H.n[1]; V.n2 = H.n[2];
  V.ncell = H.ncell;
  for (int a = 0; a < 3; ++a) V.ih2[a] = a < c->grid.dim ? (float)(1.0 / (H.h[a] * H.h[a])) : 0.0f;
  V.u = H.uf; V.ubar = H.ubarf; V.g = H.gf; V.d = H.df; V.Kc = H.Kcf;
  V.p1 = c->het_p1 ? H.p1f : nullptr;
  V.p2 = c->het_p2 ? H.p2f : nullptr;
  V.smax = c->sink.enabled ? H.smaxf : nullptr;
  V.psi0 = H.psi0f;
  for (int f = 0; f < 6; ++f) V.kb[f] = H.kbf[f];
  V.mat = c->layered ? H.mat : nullptr;
  V.cs = H.cs;
  return V;
}

// FP32 copy of a level's per-cell parameter array, in the level's layout
void to_float_at(richards_ctx* c, int l, const double* src, float* dst) {
  const HLevel& H = c->L[l];
  if (H.cs) rich::to_float_level(src, dst, H.n[0], H.n[1], H.n[2], 1, c->s);
  else rich::to_float(src, dst, H.ncell, c->s);
}

Xfer<double> xfer64(const richards_ctx* c, int l) {
  const HLevel& H = c->L[l];
  Xfer<double> X{};
  for (int a = 0; a < 3; ++a) {
    X.pc[a] = H.pc[a]; X.pj[a] = H.pj[a]; X.pw[a] = H.pw[a];
    X.rc[a] = H.rc[a]; X.ri[a] = H.ri[a]; X.rw[a] = H.rw[a];
  }
  return X;
}

Xfer<float> xfer32(const richards_ctx* c, int l) {
  const HLevel& H = c->L[l];
  Xfer<float> X{};
  for (int a = 0; a < 3; ++a) {
    X.pc[a] = H.pc[a]; X.pj[a] = H.pj[a]; X.pw[a] = H.pwf[a];
    X.rc[a] = H.rc[a]; X.ri[a] = H.ri[a]; X.rw[a] = H.rwf[a];
  }
  return X;
}

template <typename T>
Phys<T> phys(const richards_ctx* c) {
  Phys<T> P{};
  P.a = (T)c->a;
  P.xi = (T)c->opts.xi;
  P.kappa = (T)(c->opts.kappa_mode == 0 ? c->opts.kappa : 0.0);
  P.ts = (T)c->soil.theta_s;
  P.tr = (T)c->soil.theta_r;
  P.p1 = (T)c->soil.p1; P.p2 = (T)c->soil.p2; P.p3 = (T)c->soil.p3; P.p4 = (T)c->soil.p4;
  P.h1 = (T)c->sink.h1; P.h2 = (T)c->sink.h2; P.h3 = (T)c->sink.h3; P.h4 = (T)c->sink.h4;
  P.newton_k = c->opts.newton_iters;
  P.sink = c->sink.enabled;
  P.lag = c->opts.bdf2_lag;
  if (c->layered) {
    if constexpr (std::is_same<T, double>::value) P.mats = c->dmat64;
    else P.mats = c->dmat32;
    P.ddmats = c->dmatdd;
  }
  return P;
}

// fine material index for the preparation kernels (null unless layered)
const uint8_t* fine_mat(const richards_ctx* c) { return c->layered ? c->L[0].mat : nullptr; }

// m = 1 - 1/n per cell of a van Genuchten n field (null otherwise)
const double* fine_vgm(const richards_ctx* c) {
  return !c->layered && c->soil.model == RICH_VANGENUCHTEN && c->het_p2 ? c->L[0].vgm : nullptr;
}

// upload the level views and transfer tables the coarse-tail kernel reads
richards_status upload_views(richards_ctx* c) {
  std::vector<Level<double>> v64(c->nlev);
  std::vector<Xfer<double>> x64(c->nlev);
  std::vector<Level<float>> v32(c->nlev);
  std::vector<Xfer<float>> x32(c->nlev);
  for (int l = 0; l < c->nlev; ++l) {
    v64[l] = view64(c, l);
    x64[l] = xfer64(c, l);
    v32[l] = view32(c, l);
    x32[l] = xfer32(c, l);
  }
  CK(cudaMemcpyAsync(c->dL64, v64.data(), sizeof(Level<double>) * c->nlev, cudaMemcpyHostToDevice, c->s));
  CK(cudaMemcpyAsync(c->dX64, x64.data(), sizeof(Xfer<double>) * c->nlev, cudaMemcpyHostToDevice, c->s));
  CK(cudaMemcpyAsync(c->dL32, v32.data(), sizeof(Level<float>) * c->nlev, cudaMemcpyHostToDevice, c->s));
  CK(cudaMemcpyAsync(c->dX32, x32.data(), sizeof(Xfer<float>) * c->nlev, cudaMemcpyHostToDevice, c->s));
  CK(cudaStreamSynchronize(c->s));
  return RICH_OK;
}

richards_status check_launch(richards_ctx* c) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return fail(c, RICH_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e) +
                                   (c->graph_err.empty() ? "" : " (graphs: " + c->graph_err + ")"));
  return RICH_OK;
}

// ||.||_inf of a freshly computed defect (slot k of the scratch area)
richards_status read_norm(richards_ctx* c, int k, double* out, bool fp32) {
  CK(cudaMemcpyAsync(c->hscratch + k, c->scratch + k, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->s));
  CK(cudaStreamSynchronize(c->s));
  graph_harvest(c);
  const unsigned long long b = c->hscratch[k];
  if (fp32) {
    unsigned u = (unsigned)b;
    float f;
    std::memcpy(&f, &u, 4);
    *out = (double)f;
  } else {
    std::memcpy(out, &b, 8);
  }
  return RICH_OK;
}

richards_status norm64(richards_ctx* c, int l, double* out) {
  CK(cudaMemsetAsync(c->scratch, 0, sizeof(unsigned long long), c->s));
  {
    Prof pr(c, "residual64", l, c->L[l].ncell);
    rich::residual64(view64(c, l), phys<double>(c), c->soil.model, c->scratch, c->s);
  }
  TRY(check_launch(c));
  return read_norm(c, 0, out, false);
}

// NVTX range per level around that level's own launches (a profiler can then
// select the kernels of one level)
const char* level_range(int l) {
  static const char* names[] = {"L0", "L1", "L2", "L3", "L4", "L5", "L6", "L7", "L8", "L9", "L10", "L11",
                                "L12", "L13", "L14", "L15", "L16", "L17", "L18", "L19", "L20", "L21", "L22", "L23"};
  return names[l < 24 ? l : 23];
}

// coarse-grid visits from level l (cycle_gamma above gamma_levels, else 1)
int gamma_at(const richards_ctx* c, int l) {
  return (c->opts.gamma_levels <= 0 || l < c->opts.gamma_levels) ? c->opts.cycle_gamma : 1;
}

// nu NGS sweeps on a grid level: red then black half-sweeps, or, with
// ordering 0, the paper's lexicographic sweep (one launch per hyperplane;
// timed as one record per sweep)
void smooth64(richards_ctx* c, const Level<double>& F, const Phys<double>& P, int l, int nu) {
  const int model = c->soil.model;
  const long long half = (F.ncell + 1) / 2;
  for (int k = 0; k < nu; ++k) {
    if (c->opts.ordering == 0) {
      Prof pr(c, "sweep_lex64", l, F.ncell);
      rich::sweep_lex64(F, P, model, c->s);
      continue;
    }
    { Prof pr(c, "sweep64", l, half); rich::sweep64(F, P, model, 0, c->s); }
    { Prof pr(c, "sweep64", l, F.ncell - half); rich::sweep64(F, P, model, 1, c->s); }
  }
  c->updates_host += (long long)nu * F.ncell;
}

int planes_at(const richards_ctx* c, int l) { return c->tune_planes[l] > 0 ? c->tune_planes[l] : c->opts.sweep_planes; }

void smooth32(richards_ctx* c, const Level<float>& F, const Phys<float>& P, int l, int nu) {
  const int model = c->soil.model;
  const long long half = (F.ncell + 1) / 2;
  const int pl = planes_at(c, l), bx = c->tune_bx[l];
  for (int k = 0; k < nu; ++k) {
    if (c->opts.ordering == 0) {
      Prof pr(c, "sweep_lex32", l, F.ncell);
      rich::sweep_lex32(F, P, model, c->s);
      continue;
    }
    { Prof pr(c, "sweep32", l, half); rich::sweep32(F, P, model, 0, pl, c->s, bx); }
    { Prof pr(c, "sweep32", l, F.ncell - half); rich::sweep32(F, P, model, 1, pl, c->s, bx); }
  }
  c->updates_host += (long long)nu * F.ncell;
}

// ------------------------------------------------------------------------
// One V-cycle (Section 3.2, steps 1-7 with the coarse solve replaced by the
// recursion) from level l: grid kernels down to the coarse tail, which runs
// in one thread block.
// ------------------------------------------------------------------------
// d_ready: as for vcycle32 (nu1 = 0 and the finest defect already current)
void vcycle64(richards_ctx* c, int l, bool d_ready = false) {
  const int model = c->soil.model;
  const Phys<double> P = phys<double>(c);
  if (l >= c->tail_start) {
    Prof pr(c, "tail64", l, c->L[l].ncell);
    rich::tail64(c->dL64, c->dX64, l, c->nlev, P, model, c->opts.nu1, c->opts.nu2, c->opts.coarse_max_sweeps,
                 c->opts.coarse_rtol, c->opts.cycle_gamma, c->opts.gamma_levels, c->scratch + 16, c->opts.ordering,
                 c->s);
    return;
  }
  const Level<double> F = view64(c, l), C = view64(c, l + 1);
  nvtxRangePushA(level_range(l));
  smooth64(c, F, P, l, c->opts.nu1);
  if (!(d_ready && c->opts.nu1 == 0)) {
    Prof pr(c, "residual64", l, F.ncell);
    rich::residual64(F, P, model, nullptr, c->s);
  }
  { Prof pr(c, "restrict64", l, C.ncell); rich::restrict64(F, C, xfer64(c, l), F.u, F.d, C.ubar, C.d, c->s); }
  { Prof pr(c, "tau64", l + 1, C.ncell); rich::tau64(C, P, model, c->s); }
  nvtxRangePop();
  for (int q = 0; q < gamma_at(c, l); ++q) vcycle64(c, l + 1);
  nvtxRangePushA(level_range(l));
  { Prof pr(c, "prolong64", l, F.ncell); rich::prolong64(F, C, xfer64(c, l), c->s); }
  smooth64(c, F, P, l, c->opts.nu2);
  nvtxRangePop();
}

// d_ready: the finest level's defect array already holds g - N(u) for the
// current u (only used with nu1 = 0, where no pre-smoothing changes u
// between the inner stop test's defect and this cycle's restriction)
// fuse (finest level only): the last half-sweep of the post-smoothing also
// writes its cells' defects, a defect pass over the other colour completes
// d, and ||d||_inf lands in scratch slot 1, ready for the inner stop test
void vcycle32(richards_ctx* c, int l, bool d_ready = false, bool fuse = false) {
  const int model = c->soil.model;
  const Phys<float> P = phys<float>(c);
  if (l >= c->coop_start && l < c->tail_start && c->opts.ordering == 1) {
    if (!c->coop_blocks) {
      const long long need = (c->L[l].ncell / 2 + rich::COOP_THREADS - 1) / rich::COOP_THREADS;
      c->coop_blocks = (int)std::max(1LL, std::min<long long>(rich::coop_max_blocks32(model), need));
    }
    Prof pr(c, "coop32", l, c->L[l].ncell);
    const cudaError_t e = rich::coop32(c->dL32, c->dX32, l, c->nlev, c->tail_start, P, model, c->opts.nu1,
                                       c->opts.nu2, c->opts.coarse_max_sweeps, (float)c->opts.coarse_rtol,
                                       c->opts.cycle_gamma, c->opts.gamma_levels, c->scratch + 16, c->scratch + 64,
                                       c->coop_blocks, c->s);
    if (e == cudaSuccess) return;
    cudaGetLastError();                 // no cooperative launch here: the stage launches below instead
    c->graph_err = std::string("cooperative launch: ") + cudaGetErrorString(e);
    c->coop_start = MAXLEV;
  }
  if (l >= c->tail_start) {
    Prof pr(c, "tail32", l, c->L[l].ncell);
    rich::tail32(c->dL32, c->dX32, l, c->nlev, P, model, c->opts.nu1, c->opts.nu2, c->opts.coarse_max_sweeps,
                 (float)c->opts.coarse_rtol, c->opts.cycle_gamma, c->opts.gamma_levels, c->scratch + 16,
                 c->opts.ordering, c->s);
    return;
  }
  const Level<float> F = view32(c, l), C = view32(c, l + 1);
  nvtxRangePushA(level_range(l));
  smooth32(c, F, P, l, c->opts.nu1);
  if (!(d_ready && c->opts.nu1 == 0)) {
    Prof pr(c, "residual32", l, F.ncell);
    rich::residual32(F, P, model, nullptr, c->s, c->tune_rbx[l]);
  }
  { Prof pr(c, "restrict32", l, C.ncell); rich::restrict32(F, C, xfer32(c, l), F.u, F.d, C.ubar, C.d, c->s); }
  { Prof pr(c, "tau32", l + 1, C.ncell); rich::tau32(C, P, model, c->s); }
  nvtxRangePop();
  for (int q = 0; q < gamma_at(c, l); ++q) vcycle32(c, l + 1);
  nvtxRangePushA(level_range(l));
  { Prof pr(c, "prolong32", l, F.ncell); rich::prolong32(F, C, xfer32(c, l), c->s); }
  if (fuse && l == 0 && c->opts.nu2 >= 1) {
    smooth32(c, F, P, l, c->opts.nu2 - 1);
    const long long half = (F.ncell + 1) / 2;
    { Prof pr(c, "sweep32", l, half); rich::sweep32(F, P, model, 0, planes_at(c, l), c->s, c->tune_bx[l]); }
    cudaMemsetAsync(c->scratch + 1, 0, sizeof(unsigned long long), c->s);
    { Prof pr(c, "sweep_resid32", l, F.ncell - half); rich::sweep_resid32(F, P, model, c->scratch + 1, c->s); }
    { Prof pr(c, "residual32", l, half); rich::residual_color32(F, P, model, 0, c->scratch + 1, c->s); }
    c->updates_host += F.ncell;
  } else {
    smooth32(c, F, P, l, c->opts.nu2);
  }
  nvtxRangePop();
}

// One FP32 inner cycle, replayed from a CUDA graph when the options ask for it
// and the stream can be captured; the graph is captured again when a, the
// profiling state or any set-up call changed what its launches bake in.
// With nu1 = 0 and the inner stop test on, every inner cycle starts from a
// finest-level defect that is already in place: the stop test's after each
// cycle, and g itself before the first one (N(0) = 0 exactly: every
// increment of the correction equation vanishes at delta = 0).  The cycle
// then skips recomputing it.
bool top_defect_ready(const richards_ctx* c) { return c->opts.nu1 == 0 && c->opts.inner_rtol > 0.0; }

// the stop test's defect then also comes from the cycle's last half-sweep
// (see vcycle32), on levels the pipelined half-sweep serves
bool fuse_defect(const richards_ctx* c) {
  return top_defect_ready(c) && c->opts.ordering == 1 && c->opts.nu2 >= 1 && c->tail_start > 0 &&
         rich::resid_fusable32(view32(c, 0), planes_at(c, 0));
}

void run_cycle32(richards_ctx* c) {
  const bool ready = top_defect_ready(c), fuse = fuse_defect(c);
  if (c->opts.graphs && c->graphs_ok && c->s != nullptr) {
    richards_ctx::GraphRec& G = c->graphs[c->scheme_used];
    if (!G.exec || G.a != c->a || G.with_prof != c->prof) {
      if (G.exec) cudaGraphExecDestroy(G.exec);
      G.exec = nullptr;
      for (auto& r : G.prof)
        if (r.a) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
      G.prof.clear();
      const long long before = c->updates_host;
      c->capture_recs.clear();
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamBeginCapture(c->s, cudaStreamCaptureModeThreadLocal);
      const char* where = "cudaStreamBeginCapture";
      if (e == cudaSuccess) {
        c->capturing = true;
        vcycle32(c, 0, ready, fuse);
        c->capturing = false;
        const cudaError_t el = cudaGetLastError();
        e = cudaStreamEndCapture(c->s, &g);
        where = "cudaStreamEndCapture";
        if (e == cudaSuccess && el != cudaSuccess) { e = el; where = "launch during capture"; }
      }
      if (e == cudaSuccess) {
        e = cudaGraphInstantiate(&G.exec, g, 0);
        where = "cudaGraphInstantiate";
      }
      if (g) cudaGraphDestroy(g);
      const bool ok = e == cudaSuccess;
      if (!ok) c->graph_err = std::string(where) + ": " + cudaGetErrorString(e);
      G.updates = c->updates_host - before;
      c->updates_host = before;
      G.prof.swap(c->capture_recs);
      if (!ok) {                        // no graphs on this context: launch directly
        cudaGetLastError();
        for (auto& r : G.prof)
          if (r.a) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
        G.prof.clear();
        G.exec = nullptr;
        c->graphs_ok = false;
        vcycle32(c, 0, ready, fuse);
        return;
      }
      G.a = c->a;
      G.with_prof = c->prof;
    }
    if (c->harvest) {                   // the replay reuses the event nodes: read the last one first
      cudaStreamSynchronize(c->s);
      graph_harvest(c);
    }
    const cudaError_t e = cudaGraphLaunch(G.exec, c->s);
    if (e != cudaSuccess) c->graph_err = std::string("cudaGraphLaunch: ") + cudaGetErrorString(e);
    c->updates_host += G.updates;
    if (c->prof && !G.prof.empty()) c->harvest = &G;
    return;
  }
  vcycle32(c, 0, ready, fuse);
}

// ---------------------------------------------------------------------------
// The FP32 inner solve as one graph: a conditional while node whose body is
// the inner cycle, its stop test (the defect norm into scratch slot 1) and
// k_inner_loop_cond, which counts the cycle and continues while the count is
// below inner_cycles and the defect above its target -- the loop of
// step_mixed, decided on the device instead of after a host round trip per
// cycle.  The loop's control words sit in scratch slots LOOP_SLOT.. (count,
// cap, target bits, test flag), staged through the same slots of hscratch.
// ---------------------------------------------------------------------------
// finest levels of at least this many cells run their inner cycles as
// richards_step does, on their own stream, under a batcher too
constexpr long long BATCH_OWN_CELLS = 1LL << 20;

constexpr int LOOP_SLOT = 67;     // 67..70 on the device; 71 receives the count on the host

__global__ void k_inner_loop_cond(cudaGraphConditionalHandle h, const unsigned long long* nrm,
                                  unsigned long long* ctl) {
  const unsigned long long k = ++ctl[0];
  bool more = k < ctl[1];
  if (more && ctl[3]) {
    const float f = __uint_as_float((unsigned)*nrm);
    more = !((double)f <= __longlong_as_double((long long)ctl[2]));
  }
  cudaGraphSetConditional(h, more ? 1u : 0u);
}

// builds the loop graph of the current scheme and a; false when the device
// or the driver refuses it (loop_ok is then cleared: host loop from then on)
bool build_inner_loop(richards_ctx* c, richards_ctx::LoopRec& G) {
  const bool ready = top_defect_ready(c), fuse = fuse_defect(c);
  const bool test = c->opts.inner_rtol > 0.0;
  cudaGraph_t g = nullptr;
  cudaGraphConditionalHandle h = 0;
  cudaGraphNodeParams np{};
  cudaGraphNode_t node = nullptr;
  const char* where = "cudaGraphCreate";
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e == cudaSuccess) {
    where = "cudaGraphConditionalHandleCreate";
    e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
  }
  if (e == cudaSuccess) {
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    where = "cudaGraphAddNode";
    e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
  }
  const long long before = c->updates_host;
  // the body's launches are listed as a count-only profile would list them
  // (that profile adds no nodes), for richards_profile's counts
  const int prof_saved = c->prof;
  c->prof = 3;
  c->capture_recs.clear();
  if (e == cudaSuccess) {
    cudaGraph_t body = np.conditional.phGraph_out[0];
    where = "cudaStreamBeginCaptureToGraph";
    e = cudaStreamBeginCaptureToGraph(c->s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      c->capturing = true;
      vcycle32(c, 0, ready, fuse);
      G.updates = c->updates_host - before;
      if (test && !fuse) {
        cudaMemsetAsync(c->scratch + 1, 0, sizeof(unsigned long long), c->s);
        Prof pr(c, "residual32", 0, c->L[0].ncell);
        rich::residual32(view32(c, 0), phys<float>(c), c->soil.model, c->scratch + 1, c->s, c->tune_rbx[0]);
      }
      {
        Prof pr(c, "inner_loop_cond", 0, 1);
        k_inner_loop_cond<<<1, 1, 0, c->s>>>(h, c->scratch + 1, c->scratch + LOOP_SLOT);
      }
      c->capturing = false;
      const cudaError_t el = cudaGetLastError();
      cudaGraph_t out = nullptr;
      e = cudaStreamEndCapture(c->s, &out);
      where = "cudaStreamEndCapture";
      if (e == cudaSuccess && el != cudaSuccess) { e = el; where = "launch during capture"; }
    }
  }
  c->updates_host = before;
  c->prof = prof_saved;
  G.recs.swap(c->capture_recs);
  c->capture_recs.clear();
  if (e == cudaSuccess) {
    where = "cudaGraphInstantiate";
    e = cudaGraphInstantiate(&G.exec, g, 0);
  }
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    G.exec = nullptr;
    c->loop_ok = false;
    c->loop_err = std::string(where) + ": " + cudaGetErrorString(e);
    return false;
  }
  G.a = c->a;
  return true;
}

// whether the inner solve runs as the loop graph (graphs on, no timing, no
// cooperative levels, a stream of the context's own)
bool inner_loop_usable(const richards_ctx* c) {
  return c->opts.graphs && c->graphs_ok && c->loop_ok && c->s != nullptr && (c->prof == 0 || c->prof == 3) &&
         !c->capturing &&
         c->coop_start >= c->nlev && c->opts.inner_cycles >= 1;
}

// one inner solve through the loop graph: at most inner_cycles cycles, until
// the defect norm is at most target (test: inner_rtol > 0); *cycles gets the
// count.  RICH_EINVAL (nothing launched) when the graph cannot be built.
richards_status run_inner_loop(richards_ctx* c, double target, int* cycles) {
  richards_ctx::LoopRec& G = c->loops[c->scheme_used];
  if (!G.exec || G.a != c->a) {
    if (G.exec) cudaGraphExecDestroy(G.exec);
    G.exec = nullptr;
    if (!build_inner_loop(c, G)) return RICH_EINVAL;
  }
  unsigned long long* h = c->hscratch + LOOP_SLOT;
  h[0] = 0;
  h[1] = (unsigned long long)c->opts.inner_cycles;
  std::memcpy(&h[2], &target, sizeof(double));
  h[3] = c->opts.inner_rtol > 0.0 ? 1ull : 0ull;
  CK(cudaMemcpyAsync(c->scratch + LOOP_SLOT, h, 4 * sizeof(unsigned long long), cudaMemcpyHostToDevice, c->s));
  CK(cudaGraphLaunch(G.exec, c->s));
  CK(cudaMemcpyAsync(c->hscratch + LOOP_SLOT + 4, c->scratch + LOOP_SLOT, sizeof(unsigned long long),
                     cudaMemcpyDeviceToHost, c->s));
  CK(cudaStreamSynchronize(c->s));
  *cycles = (int)c->hscratch[LOOP_SLOT + 4];
  c->updates_host += (long long)*cycles * G.updates;
  if (c->prof == 3)                     // counted launches: the body's, once per pass
    for (int k = 0; k < *cycles; ++k)
      for (const auto& r : G.recs) prof_count(c, r.name, r.level, r.cells);
  return RICH_OK;
}

// coarse copies of the lagged conductivity and boundary conductances
// (mixed mode: the coarse coefficients only feed the FP32 inner cycles, so
// they are restricted in FP32 from the finest level's FP32 copies)
richards_status restrict_coefficients(richards_ctx* c) {
  Prof pr(c, "coefficients", 0, c->L[0].ncell);
  if (c->opts.precision >= 1) {
    for (int f = 0; f < 2 * c->grid.dim; ++f) rich::to_float(c->L[0].kb[f], c->L[0].kbf[f], c->L[0].nface[f], c->s);
    for (int l = 0; l + 1 < c->nlev; ++l) {
      const Level<float> F = view32(c, l), C = view32(c, l + 1);
      rich::restrict32(F, C, xfer32(c, l), c->L[l].Kcf, nullptr, c->L[l + 1].Kcf, nullptr, c->s);
      for (int f = 0; f < 2 * c->grid.dim; ++f)
        rich::restrict_face32(geom(c, l), geom(c, l + 1), xfer32(c, l), f / 2, c->L[l].kbf[f], c->L[l + 1].kbf[f],
                              c->s);
    }
    return check_launch(c);
  }
  for (int l = 0; l + 1 < c->nlev; ++l) {
    const Level<double> F = view64(c, l), C = view64(c, l + 1);
    rich::restrict64(F, C, xfer64(c, l), c->L[l].Kc, nullptr, c->L[l + 1].Kc, nullptr, c->s);
    for (int f = 0; f < 2 * c->grid.dim; ++f)
      rich::restrict_face64(geom(c, l), geom(c, l + 1), xfer64(c, l), f / 2, c->L[l].kb[f], c->L[l + 1].kb[f], c->s);
  }
  return check_launch(c);
}

richards_status do_prepare(richards_ctx* c, double dt, int scheme) {
  c->bp = BatchProgress{};                 // a batched step in progress restarts
  if (!c->soil_set) return fail(c, RICH_EINVAL, "soil not set");
  if (!c->bc_set) return fail(c, RICH_EINVAL, "boundary conditions not set");
  if (!c->have_state) return fail(c, RICH_EINVAL, "state not set");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, RICH_EINVAL, "dt must be positive and finite");
  if (scheme != 1 && scheme != 2) return fail(c, RICH_EINVAL, "scheme must be 1 (BDF1) or 2 (BDF2)");
  if (scheme == 2 && !c->have_prev) scheme = 1;
  c->scheme_used = scheme;
  c->dt = dt;
  c->a = scheme == 1 ? 1.0 / dt : 1.5 / dt;
  const Phys<double> P = phys<double>(c);
  HLevel& F = c->L[0];
  Prof pr(c, "prep", 0, F.ncell);
  const bool cache = c->opts.precision >= 1;
  const bool dd = c->opts.precision == 1;   // float-float outer layer; else FP64
  if (c->opts.precision == 2)   // FP64-outer mixed mode: FP64 laws, FP64 theta caches, FP32 copy of Kc
    rich::prep_lagged(geom(c, 0), c->psi_n, c->psi_nm1, c->het_Ks ? c->Ks : nullptr, c->soil.Ks,
                      c->het_p1 ? F.p1 : nullptr, c->het_p2 ? F.p2 : nullptr, fine_mat(c), P, c->soil.model, scheme,
                      dt, F.Kc, F.Kcf, F.g, F.u, c->th_n_valid ? c->th_n : nullptr,
                      c->th_nm1_valid ? c->th_nm1 : nullptr, c->th_n_valid ? nullptr : c->th_n,
                      c->th_nm1_valid ? nullptr : c->th_nm1, c->opts.predictor == 1, c->s, fine_vgm(c));
  else if (dd)    // mixed mode: float-float arithmetic, theta caches
    rich::prep_lagged_dd(geom(c, 0), c->psi_n, c->psi_nm1, c->het_Ks ? c->Ks : nullptr, c->soil.Ks,
                         c->het_p1 ? F.p1 : nullptr, c->het_p2 ? F.p2 : nullptr, fine_mat(c), P, rich::make_ddphys(P),
                         c->soil.model, scheme, dt, F.Kc, F.Kcf, F.g, F.u, c->th_n_valid ? c->th_n : nullptr,
                         c->th_nm1_valid ? c->th_nm1 : nullptr, c->th_n_valid ? nullptr : c->th_n,
                         c->th_nm1_valid ? nullptr : c->th_nm1, c->opts.predictor == 1, c->s);
  else
    rich::prep_lagged(geom(c, 0), c->psi_n, c->psi_nm1, c->het_Ks ? c->Ks : nullptr, c->soil.Ks,
                      c->het_p1 ? F.p1 : nullptr, c->het_p2 ? F.p2 : nullptr, fine_mat(c), P, c->soil.model, scheme,
                      dt, F.Kc, nullptr, F.g, F.u, nullptr, nullptr, nullptr, nullptr, false, c->s, fine_vgm(c));
  if (cache) {
    c->th_n_valid = true;
    if (scheme == 2) c->th_nm1_valid = true;
  }
  double* kbw[6];
  for (int f = 0; f < 6; ++f) kbw[f] = F.kb[f];
  if (dd)
    rich::prep_rhs_dd(geom(c, 0), c->bcdev, c->het_Ks ? c->Ks : nullptr, c->soil.Ks, c->het_p1 ? F.p1 : nullptr,
                      c->het_p2 ? F.p2 : nullptr, fine_mat(c), P, rich::make_ddphys(P), c->soil.model, F.Kc, F.g, kbw,
                      c->s);
  else
    rich::prep_rhs(geom(c, 0), c->bcdev, c->het_Ks ? c->Ks : nullptr, c->soil.Ks, c->het_p1 ? F.p1 : nullptr,
                   c->het_p2 ? F.p2 : nullptr, fine_mat(c), P, c->soil.model, F.Kc, F.g, kbw, c->s);
  TRY(check_launch(c));
  TRY(restrict_coefficients(c));
  c->prepared = true;
  return RICH_OK;
}

// the history shift of an accepted step, as copies on the context's stream
// (finish_step_launch), and what follows once they are done (finish_step_done)
richards_status finish_step_launch(richards_ctx* c, int theta_fresh) {
  if (theta_fresh == 1) {            // th_cur = theta(psi^{n+1})
    double* t = c->th_nm1;
    c->th_nm1 = c->th_n;
    c->th_n = c->th_cur;
    c->th_cur = t;
    c->th_nm1_valid = true;
  } else if (theta_fresh == 0) {     // psi^{n+1} = psi^n
    CK(cudaMemcpyAsync(c->th_nm1, c->th_n, sizeof(double) * c->L[0].ncell, cudaMemcpyDeviceToDevice, c->s));
    c->th_nm1_valid = true;
  }
  std::swap(c->psi_n, c->psi_nm1);
  CK(cudaMemcpyAsync(c->psi_n, c->L[0].u, sizeof(double) * c->L[0].ncell, cudaMemcpyDeviceToDevice, c->s));
  return RICH_OK;
}

richards_status finish_step_done(richards_ctx* c, richards_status st) {
  c->have_prev = true;
  c->t += c->dt;
  if (st != RICH_OK) return fail(c, st, "no convergence within the cycle limit");
  return RICH_OK;
}

richards_status finish_step(richards_ctx* c, double r, richards_status st, int theta_fresh = -1) {
  if (std::isnan(r)) return fail(c, RICH_ENAN, "NaN in the iterate; state kept at psi^n");
  TRY(finish_step_launch(c, theta_fresh));
  CK(cudaStreamSynchronize(c->s));
  return finish_step_done(c, st);
}

richards_status read_stats(richards_ctx* c, long long* tail_updates) {
  CK(cudaMemcpyAsync(c->hscratch + 16, c->scratch + 16, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->s));
  CK(cudaStreamSynchronize(c->s));
  *tail_updates = (long long)c->hscratch[16];
  return RICH_OK;
}

// The water balance in two halves: its launches and copies to the host on
// the context's stream (*nb_out: partial sums; 0 when r is not finite), and
// the sums once the stream is done (water_balance_done).
richards_status water_balance_launch(richards_ctx* c, double r, const double* th_new, const double* th_n,
                                     const double* th_nm1, int* nb_out) {
  *nb_out = 0;
  if (!std::isfinite(r)) return RICH_OK;
  unsigned* dmin = (unsigned*)(c->mass_part + MASS_PARTS);
  CK(cudaMemsetAsync(dmin, 0xff, sizeof(unsigned), c->s));
  int nb;
  {
    Prof pr(c, "mass_balance", 0, c->L[0].ncell);
    nb = rich::mass_balance(view64(c, 0), geom(c, 0), c->bcdev, phys<double>(c), phys<float>(c), c->soil.model,
                            c->psi_n, c->psi_nm1, c->scheme_used, c->dt, th_new, th_n,
                            c->scheme_used == 2 ? th_nm1 : nullptr, c->mass_part, dmin, c->opts.precision != 1, c->s);
  }
  TRY(check_launch(c));
  if (nb > MASS_PARTS) return fail(c, RICH_ECUDA, "water balance: too many blocks");
  CK(cudaMemcpyAsync(c->hmass, c->mass_part, sizeof(double) * nb, cudaMemcpyDeviceToHost, c->s));
  CK(cudaMemcpyAsync(c->hmass + MASS_PARTS, dmin, sizeof(unsigned), cudaMemcpyDeviceToHost, c->s));
  *nb_out = nb;
  return RICH_OK;
}

void water_balance_done(richards_ctx* c, double r, int nb, richards_step_info* info) {
  info->mass_defect = NAN;
  info->err_bound = NAN;
  if (nb <= 0) return;
  long double sum = 0.0L;
  for (int b = 0; b < nb; ++b) sum += (long double)c->hmass[b];
  info->mass_defect = (double)(sum / (long double)c->a);
  unsigned bits;
  std::memcpy(&bits, c->hmass + MASS_PARTS, sizeof(unsigned));
  float dm;
  std::memcpy(&dm, &bits, sizeof(float));
  const double nrm = r * c->a;      // ||N(psi) - g||_inf
  info->err_bound = (bits < 0x7f800000u && dm > 0.0f) ? nrm / (double)dm : INFINITY;
}

// Water balance and error bound of the iterate about to be accepted (before
// the history shift); r = tau_eff ||g - N(psi)||_inf.  th_*: theta caches
// (nullable: evaluated).  FP64 laws and sums, except in the float-float
// mixed mode (precision 1).
richards_status water_balance(richards_ctx* c, double r, richards_step_info* info, const double* th_new,
                              const double* th_n, const double* th_nm1) {
  if (!info) return RICH_OK;
  int nb = 0;
  TRY(water_balance_launch(c, r, th_new, th_n, th_nm1, &nb));
  if (nb > 0) CK(cudaStreamSynchronize(c->s));
  water_balance_done(c, r, nb, info);
  return RICH_OK;
}

// Full multigrid pass (Section 3.2: coarsest grid first, the solution
// interpolated to successively finer grids, fmg_cycles cycles on each).
// Coarse right sides and starting iterates are the restricted finer ones
// (ubar keeps the restricted iterate); prolong() then adds
// P(coarse iterate - ubar) to the finer iterate.  FP64 levels (FP64 mode).
void fmg64(richards_ctx* c) {
  const int nl = c->nlev;
  if (nl < 2 || c->opts.fmg_cycles <= 0) return;
  for (int l = 0; l + 1 < nl; ++l) {
    HLevel &F = c->L[l], &C = c->L[l + 1];
    {
      Prof pr(c, "fmg_restrict64", l, C.ncell);
      rich::restrict64(view64(c, l), view64(c, l + 1), xfer64(c, l), F.u, F.g, C.ubar, C.g, c->s);
    }
    cudaMemcpyAsync(C.u, C.ubar, sizeof(double) * C.ncell, cudaMemcpyDeviceToDevice, c->s);
  }
  for (int k = 0; k < c->opts.fmg_cycles; ++k) vcycle64(c, nl - 1);
  for (int l = nl - 2; l >= 0; --l) {
    {
      Prof pr(c, "prolong64", l, c->L[l].ncell);
      rich::prolong64(view64(c, l), view64(c, l + 1), xfer64(c, l), c->s);
    }
    for (int k = 0; k < c->opts.fmg_cycles; ++k) vcycle64(c, l);
  }
}

// The same pass on the FP32 correction problem of the mixed mode (finest
// level: delta = 0, right side the outer defect).
void fmg32(richards_ctx* c) {
  const int nl = c->nlev;
  if (nl < 2 || c->opts.fmg_cycles <= 0) return;
  for (int l = 0; l + 1 < nl; ++l) {
    HLevel &F = c->L[l], &C = c->L[l + 1];
    {
      Prof pr(c, "fmg_restrict32", l, C.ncell);
      rich::restrict32(view32(c, l), view32(c, l + 1), xfer32(c, l), F.uf, F.gf, C.ubarf, C.gf, c->s,
                       F.cs ? 2 : 0);
    }
    cudaMemcpyAsync(C.uf, C.ubarf, sizeof(float) * C.ncell, cudaMemcpyDeviceToDevice, c->s);
  }
  for (int k = 0; k < c->opts.fmg_cycles; ++k) vcycle32(c, nl - 1);
  for (int l = nl - 2; l >= 0; --l) {
    {
      Prof pr(c, "prolong32", l, c->L[l].ncell);
      rich::prolong32(view32(c, l), view32(c, l + 1), xfer32(c, l), c->s);
    }
    for (int k = 0; k < c->opts.fmg_cycles; ++k) vcycle32(c, l);
  }
}

richards_status step_fp64(richards_ctx* c, richards_step_info* info) {
  const double teff = 1.0 / c->a;
  double nrm;
  TRY(norm64(c, 0, &nrm));
  double r = teff * nrm;
  const double r0 = r;
  int cycles = 0, fmg = 0;                            // cycles after / in the FMG pass
  if (c->opts.fmg_cycles > 0 && c->nlev > 1) {      // full multigrid start
    fmg64(c);
    TRY(check_launch(c));
    fmg = c->opts.fmg_cycles;
    TRY(norm64(c, 0, &nrm));
    r = teff * nrm;
  }
  // every cycle follows a norm64 of the current iterate, whose defect the
  // cycle reuses when there is no pre-smoothing
  while (!(r <= c->opts.tol) && cycles < c->opts.max_cycles && !std::isnan(r)) {
    vcycle64(c, 0, true);
    TRY(check_launch(c));
    ++cycles;
    TRY(norm64(c, 0, &nrm));
    r = teff * nrm;
  }
  long long tu = 0;
  TRY(read_stats(c, &tu));
  if (info) {
    info->cycles = cycles + fmg;
    info->outer_iters = 0;
    info->scheme_used = c->scheme_used;
    info->resid0 = r0;
    info->resid = r;
    info->cell_updates = c->updates_host + tu;
  }
  TRY(water_balance(c, r, info, nullptr, nullptr, nullptr));
  return finish_step(c, r, r <= c->opts.tol ? RICH_OK : RICH_ENOCONV);
}

// Mixed precision: defect r = g - N(psi) in float-float arithmetic (~1e-12
// relative, no FP64 instruction); FP32 FAS cycles on the correction
// equation N(psi + delta) - N(psi) = r; psi += delta (FP64); repeat until the
// stop test on ||r|| holds.  precision 2 (FP64 outer): the system (lagged K,
// history, right side) is the FP64 one, the float-float defects only steer
// the corrections, and the defect that decides the stop test -- computed
// whenever a float-float defect passes it, or the outer limit is reached --
// is FP64; it also gives theta(psi^{n+1}) to the FP64 history cache.
// The outer defect of the mixed mode (float-float, or FP64 with fp64) into
// the inner problem's right side, frozen state and zero correction, with
// ||d||_inf in scratch slot 0.  cached: the iterate is psi^n, whose theta is
// cached; otherwise theta of the iterate goes to th_cur (FP64 outer: only
// from the FP64 defect).
richards_status outer_defect_launch(richards_ctx* c, bool cached, bool fp64) {
  HLevel& F = c->L[0];
  const Phys<double> P64 = phys<double>(c);
  CK(cudaMemsetAsync(c->scratch, 0, sizeof(unsigned long long), c->s));
  double* th_out = cached || (c->opts.precision == 2 && !fp64) ? nullptr : c->th_cur;
  if (fp64) {
    Prof pr(c, "outer_residual64", 0, F.ncell);
    rich::outer_residual64(view64(c, 0), P64, c->soil.model, F.gf, F.psi0f, F.uf, c->scratch,
                           cached ? c->th_n : nullptr, th_out, F.cs, c->s, fine_vgm(c));
  } else {
    Prof pr(c, "outer_residual", 0, F.ncell);
    rich::outer_residual_dd(view64(c, 0), P64, rich::make_ddphys(P64), c->soil.model, F.gf, F.psi0f, F.uf,
                            c->scratch, cached ? c->th_n : nullptr, th_out, F.cs, c->s);
  }
  return check_launch(c);
}

// the finest defect of the inner problem at delta = 0, which is g (natural
// layout, whatever g's)
richards_status defect_from_g(richards_ctx* c) {
  HLevel& F = c->L[0];
  if (F.cs) rich::cs_to_natural(F.gf, F.df, F.n[0], F.n[1], F.n[2], c->s);
  else CK(cudaMemcpyAsync(F.df, F.gf, sizeof(float) * F.ncell, cudaMemcpyDeviceToDevice, c->s));
  return check_launch(c);
}

// the coarse copies of the inner problem's frozen state psi0
void restrict_psi0(richards_ctx* c) {
  for (int l = 0; l + 1 < c->nlev; ++l) {
    Prof pr(c, "restrict_psi0", l, c->L[l + 1].ncell);
    rich::restrict32(view32(c, l), view32(c, l + 1), xfer32(c, l), c->L[l].psi0f, nullptr, c->L[l + 1].psi0f,
                     nullptr, c->s, c->L[l].cs ? 1 : 0);
  }
}

richards_status step_mixed(richards_ctx* c, richards_step_info* info) {
  const double teff = 1.0 / c->a;
  const int model = c->soil.model;
  const Phys<float> P32 = phys<float>(c);
  HLevel& F = c->L[0];
  double r = 0.0, r0 = 0.0;
  int outer = 0, inner = 0;
  richards_status st = RICH_OK;
  // theta(psi) from the cache of theta(psi^n) before the first correction,
  // else evaluated and kept in th_cur (theta(psi^{n+1}) once accepted)
  const bool outer64 = c->opts.precision == 2;
  auto defect = [&](bool cached, bool fp64, double* out) -> richards_status {
    TRY(outer_defect_launch(c, cached, fp64));
    double nrm;
    TRY(read_norm(c, 0, &nrm, !fp64));
    *out = teff * nrm;
    return RICH_OK;
  };
  // with the predictor (BDF2 steps) the iteration starts at psi*, not psi^n
  const bool predicted = c->opts.predictor == 1 && c->scheme_used == 2;
  // FP64 outer: a float-float defect that passes the stop test, or stops
  // falling (less than halved by a correction: near tol it may sit on its own
  // rounding floor), or the outer limit hands over to FP64 defects for the
  // rest of the step
  bool use64 = false;
  double r_ff = INFINITY;
  for (;;) {
    const bool cached = outer == 0 && !predicted;
    if (!use64) {
      const double prev = r_ff;
      TRY(defect(cached, false, &r_ff));
      r = r_ff;
      use64 = outer64 && !std::isnan(r) &&
              (!(r > c->opts.tol) || outer >= c->opts.max_outer || r > 0.5 * prev);
    }
    if (use64) TRY(defect(cached, true, &r));     // the FP64 defect decides
    if (outer == 0) r0 = r;
    if (!(r > c->opts.tol) || std::isnan(r)) break;
    if (outer >= c->opts.max_outer) { st = RICH_ENOCONV; break; }
    restrict_psi0(c);
    const double rin0 = r / teff;       // ||g - N(psi)||_inf of this defect
    // an inner solve need not reduce its defect below what the stop test
    // asks of the next outer defect (with a margin of 0.3 for the FP32 and
    // nonlinear remainder): close to tol it stops early
    const double rtol_in = std::max(c->opts.inner_rtol, 0.3 * c->opts.tol / r);
    // (FP64 outer: an inner solve aimed at the stop test itself is expected
    // to pass it, so the next defect goes to FP64 straight away instead of
    // after a float-float one that would only say so)
    if (outer64 && rtol_in > c->opts.inner_rtol) use64 = true;
    bool done_in = false;
    const bool fmg_start = c->opts.fmg_cycles > 0 && c->nlev > 1;
    if (top_defect_ready(c) && !fmg_start)          // the defect at delta = 0 is g
      TRY(defect_from_g(c));
    if (fmg_start) {                                // full multigrid start of the inner solve
      fmg32(c);
      inner += c->opts.fmg_cycles;
      if (c->opts.inner_rtol > 0.0) {
        CK(cudaMemsetAsync(c->scratch + 1, 0, sizeof(unsigned long long), c->s));
        {
          Prof pr(c, "residual32", 0, F.ncell);
          rich::residual32(view32(c, 0), P32, model, c->scratch + 1, c->s, c->tune_rbx[0]);
        }
        double rin;
        TRY(read_norm(c, 1, &rin, true));
        done_in = rin <= rtol_in * rin0;
      }
    }
    const bool fused = fuse_defect(c);           // the cycle leaves d and its norm
    if (!done_in && inner_loop_usable(c)) {     // the whole inner solve on the device
      int k = 0;
      if (run_inner_loop(c, rtol_in * rin0, &k) == RICH_OK) {
        inner += k;
        done_in = true;
      }
    }
    for (int k = 0; k < c->opts.inner_cycles && !done_in; ++k) {
      run_cycle32(c);
      ++inner;
      if (c->opts.inner_rtol > 0.0 && k + 1 < c->opts.inner_cycles) {
        if (!fused) {
          CK(cudaMemsetAsync(c->scratch + 1, 0, sizeof(unsigned long long), c->s));
          Prof pr(c, "residual32", 0, F.ncell);
          rich::residual32(view32(c, 0), P32, model, c->scratch + 1, c->s, c->tune_rbx[0]);
        }
        double rin;
        TRY(read_norm(c, 1, &rin, true));
        if (rin <= rtol_in * rin0) break;
      }
    }
    {
      Prof pr(c, "apply_delta", 0, F.ncell);
      rich::apply_delta(F.u, F.uf, F.ncell, c->s);
    }
    TRY(check_launch(c));
    ++outer;
  }
  long long tu = 0;
  TRY(read_stats(c, &tu));
  if (info) {
    info->cycles = inner;
    info->outer_iters = outer;
    info->scheme_used = c->scheme_used;
    info->resid0 = r0;
    info->resid = r;
    info->cell_updates = c->updates_host + tu;
  }
  const bool moved = outer > 0 || predicted;      // theta(psi^{n+1}) is in th_cur
  TRY(water_balance(c, r, info, moved ? c->th_cur : c->th_n, c->th_n, c->th_nm1_valid ? c->th_nm1 : nullptr));
  return finish_step(c, r, st, moved ? 1 : 0);
}

}  // namespace

// ==========================================================================
// Batched steps of mixed-precision contexts (served requests), in ticks:
// every context does the next part of its own step (batch_tick); the outer
// defects and decisions of all contexts that are at one are taken together
// (one synchronisation per stream), and the FP32 inner cycles of all
// contexts in an inner solve run together, each stage of a cycle one launch
// over the descriptors of all of them (batch.cu).  The work
// of one context alone (preparation, outer defects, coarse copies of psi0,
// updates, water balance) stays on the context's own stream, so that the
// contexts' small launches overlap; events order it against the batched
// stages on the batcher's stream.
// ==========================================================================
struct richards_batcher {
  cudaStream_t s = nullptr;
  int cap = 0;                               // contexts the tables hold
  rich::BJob32* dtable = nullptr;            // cap x MAXLEV descriptors (device)
  rich::BJob32* htable = nullptr;            // staging copy (pinned)
  unsigned long long* dnorm = nullptr;       // inner-norm slot of each context (float bits; device)
  unsigned long long* hnorm = nullptr;       // pinned copy
  cudaEvent_t fork = nullptr;                // batcher stream -> context streams
  std::vector<cudaEvent_t> join;             // context stream (per slot) -> batcher stream
  std::string err;
};

namespace {

struct BatchCtx {
  richards_ctx* c = nullptr;
  int slot = 0;                              // index in this call's table and norm slots
};

int batch_nk(const richards_ctx* c) {
  const int k = c->opts.newton_iters;
  return (k == 1 || k == 2) ? k : 0;
}

// one stage over the level-l descriptors of the listed contexts, grouped by
// Newton count (the laws share a launch), at most BATCH_MAX descriptors per
// launch
void batch_stage(richards_batcher* b, std::vector<BatchCtx>& B, const std::vector<int>& who, int op, int l,
                 int color, bool with_norm) {
  std::map<int, std::vector<int>> groups;
  for (int k : who) groups[batch_nk(B[k].c)].push_back(k);
  for (auto& kv : groups) {
    const std::vector<int>& ks = kv.second;
    for (size_t a = 0; a < ks.size(); a += rich::BATCH_MAX) {
      rich::BList list{};
      list.n = 0;
      int blocks = 0;
      for (size_t q = a; q < ks.size() && q < a + rich::BATCH_MAX; ++q) {
        const int j = B[ks[q]].slot * MAXLEV + l;
        list.job[list.n] = j;
        list.block0[list.n] = blocks;
        blocks += rich::batch_blocks(op, b->htable[j]);
        ++list.n;
      }
      list.block0[list.n] = blocks;
      rich::batch32(op, kv.first, b->dtable, list, color, with_norm, b->s);
    }
  }
}

void batch_tail(richards_batcher* b, std::vector<BatchCtx>& B, const std::vector<int>& who, int l) {
  const richards_opts& o = B[who[0]].c->opts;
  for (size_t a = 0; a < who.size(); a += rich::BATCH_MAX) {
    rich::BList list{};
    for (size_t q = a; q < who.size() && q < a + rich::BATCH_MAX; ++q)
      list.job[list.n++] = B[who[q]].slot * MAXLEV + l;
    rich::batch_tail32(b->dtable, list, o.nu1, o.nu2, o.coarse_max_sweeps, (float)o.coarse_rtol, o.cycle_gamma,
                       o.gamma_levels, b->s);
  }
}

void batch_smooth(richards_batcher* b, std::vector<BatchCtx>& B, const std::vector<int>& who, int l, int nu) {
  for (int q = 0; q < nu; ++q) {
    batch_stage(b, B, who, rich::BOP_SWEEP, l, 0, false);
    batch_stage(b, B, who, rich::BOP_SWEEP, l, 1, false);
  }
  for (int k : who) B[k].c->updates_host += (long long)nu * B[k].c->L[l].ncell;
}

// vcycle32 for all listed contexts at once (top: level 0 of the inner
// solve, where a context whose stop test left the defect in place skips it)
void batch_vcycle(richards_batcher* b, std::vector<BatchCtx>& B, const std::vector<int>& who, int l, bool top) {
  std::vector<int> tail, grid;
  for (int k : who) (l >= B[k].c->tail_start ? tail : grid).push_back(k);
  if (!tail.empty()) batch_tail(b, B, tail, l);
  if (grid.empty()) return;
  const richards_opts& o = B[grid[0]].c->opts;
  batch_smooth(b, B, grid, l, o.nu1);
  std::vector<int> need;
  for (int k : grid)
    if (!(top && top_defect_ready(B[k].c) && o.nu1 == 0)) need.push_back(k);
  if (!need.empty()) batch_stage(b, B, need, rich::BOP_RESID, l, 0, false);
  batch_stage(b, B, grid, rich::BOP_RESTRICT, l, 0, false);
  batch_stage(b, B, grid, rich::BOP_TAU, l, 0, false);
  for (int q = 0; q < gamma_at(B[grid[0]].c, l); ++q) batch_vcycle(b, B, grid, l + 1, false);
  batch_stage(b, B, grid, rich::BOP_PROLONG, l, 0, false);
  batch_smooth(b, B, grid, l, o.nu2);
}

double host_norm(const richards_ctx* c, int k, bool fp32) {
  const unsigned long long bits = c->hscratch[k];
  if (fp32) {
    const unsigned u = (unsigned)bits;
    float f;
    std::memcpy(&f, &u, 4);
    return (double)f;
  }
  double d;
  std::memcpy(&d, &bits, 8);
  return d;
}

richards_status bfail(richards_batcher* b, richards_status st, const std::string& msg) {
  b->err = msg;
  return st;
}

#define TRY_B(expr)                            \
  do {                                         \
    const richards_status s_ = (expr);         \
    if (s_ != RICH_OK) return s_;              \
  } while (0)

#define BCK(call)                                                                                 \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess) return bfail(b, RICH_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// the listed contexts' streams wait for the batcher's stream
richards_status bfork(richards_batcher* b, std::vector<BatchCtx>& B, const std::vector<int>& who) {
  BCK(cudaEventRecord(b->fork, b->s));
  for (int k : who)
    if (B[k].c->s != b->s) BCK(cudaStreamWaitEvent(B[k].c->s, b->fork, 0));
  return RICH_OK;
}

// the batcher's stream waits for the listed contexts' streams
richards_status bjoin(richards_batcher* b, std::vector<BatchCtx>& B, const std::vector<int>& who) {
  for (int k : who) {
    cudaStream_t cs = B[k].c->s;
    if (cs == b->s) continue;
    BCK(cudaEventRecord(b->join[B[k].slot], cs));
    BCK(cudaStreamWaitEvent(b->s, b->join[B[k].slot], 0));
  }
  return RICH_OK;
}

// descriptors of every level of context k (its physics record carries the
// step's a = 1/dt or 3/(2 dt): rebuilt whenever the context prepares a step)
void batch_table_slot(richards_batcher* b, std::vector<BatchCtx>& B, int k) {
  richards_ctx* c = B[k].c;
  for (int l = 0; l < c->nlev; ++l) {
    rich::BJob32& J = b->htable[B[k].slot * MAXLEV + l];
    J = rich::BJob32{};
    J.F = view32(c, l);
    if (l + 1 < c->nlev) {
      J.C = view32(c, l + 1);
      J.X = xfer32(c, l);
    }
    J.P = phys<float>(c);
    J.dLs = c->dL32;
    J.dXs = c->dX32;
    J.level = l;
    J.nlev = c->nlev;
    J.model = c->soil.model;
    J.norm = b->dnorm + B[k].slot;
    J.stats = c->scratch + 16;
  }
}

// the descriptors of the listed contexts to the device (the batcher's stream
// is idle first, so that no earlier copy still reads the staging table)
richards_status batch_upload(richards_batcher* b, std::vector<BatchCtx>& B, const std::vector<int>& who) {
  if (who.empty()) return RICH_OK;
  BCK(cudaStreamSynchronize(b->s));
  for (int k : who) {
    batch_table_slot(b, B, k);
    const size_t off = (size_t)B[k].slot * MAXLEV;
    BCK(cudaMemcpyAsync(b->dtable + off, b->htable + off, sizeof(rich::BJob32) * MAXLEV, cudaMemcpyHostToDevice,
                        b->s));
  }
  return RICH_OK;
}

// One tick: every listed context does the next part of its current step
// (the same operations, in the same order, as step_mixed):
//   idle, with steps wanted  -> preparation and the first outer defect;
//   defect                   -> the outer defect (float-float, or FP64 from
//                               the point where step_mixed switches); the
//                               decision after it: the FP64 defect next,
//                               the end of the step, or an inner solve;
//   inner                    -> one FP32 V-cycle (the cycles of all such
//                               contexts as shared batched launches) and its
//                               stop test; at the end of the inner solve
//                               the correction is applied (-> defect);
//   finish                   -> water balance and history shift.
// Work of one context alone runs on its stream and overlaps the batched
// cycle on the batcher's stream; one wait per stream ends the tick.
// done[k] = 1 when context k completed a step (status in sst[k], its
// statistics in sinfo[k]).
richards_status batch_tick(richards_batcher* b, std::vector<BatchCtx>& B, const double* dt, const int* scheme,
                           const std::vector<int>& want, std::vector<char>& done, std::vector<richards_status>& sst,
                           std::vector<richards_step_info>& sinfo) {
  const int n = (int)B.size();
  std::vector<int> defect, inner, finish, own, started;
  for (int k = 0; k < n; ++k) {
    richards_ctx* c = B[k].c;
    BatchProgress& X = c->bp;
    done[k] = 0;
    if (X.phase == BP_IDLE && want[k] > 0) {
      c->updates_host = 0;
      BCK(cudaMemsetAsync(c->scratch + 16, 0, sizeof(unsigned long long), c->s));
      const richards_status sp = do_prepare(c, dt[k], scheme[k]);
      own.push_back(k);
      if (sp != RICH_OK) {                     // the step fails before it starts
        done[k] = 1;
        sst[k] = sp;
        sinfo[k] = richards_step_info{};
        continue;
      }
      X = BatchProgress{};
      X.phase = BP_DEFECT;
      X.predicted = c->opts.predictor == 1 && c->scheme_used == 2;
      started.push_back(k);
    }
    if (X.phase == BP_DEFECT) defect.push_back(k);
    else if (X.phase == BP_INNER) inner.push_back(k);
    else if (X.phase == BP_FINISH) finish.push_back(k);
  }
  TRY_B(batch_upload(b, B, started));
  // work of one context alone, on its stream
  for (int k : defect) {
    richards_ctx* c = B[k].c;
    const BatchProgress& X = c->bp;
    const richards_status sd = outer_defect_launch(c, X.outer == 0 && !X.predicted, X.use64);
    if (sd != RICH_OK) return bfail(b, sd, c->err);
    BCK(cudaMemcpyAsync(c->hscratch, c->scratch, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->s));
    own.push_back(k);
  }
  for (int k : finish) {
    richards_ctx* c = B[k].c;
    BatchProgress& X = c->bp;
    const bool moved = X.outer > 0 || X.predicted;
    X.nbal = 0;
    X.fin = cudaMemcpyAsync(c->hscratch + 16, c->scratch + 16, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                            c->s) == cudaSuccess ? RICH_OK : fail(c, RICH_ECUDA, "stats copy");
    if (X.fin == RICH_OK)
      X.fin = water_balance_launch(c, X.r, moved ? c->th_cur : c->th_n, c->th_n,
                                   c->th_nm1_valid ? c->th_nm1 : nullptr, &X.nbal);
    if (X.fin == RICH_OK && !std::isnan(X.r)) X.fin = finish_step_launch(c, moved ? 1 : 0);
    own.push_back(k);
  }
  // one FP32 V-cycle of every context in an inner solve, and the stop tests.
  // A context whose finest level has BATCH_OWN_CELLS cells or more fills the
  // GPU alone: its cycle is richards_step's (the context's cycle graph, on its
  // own stream); the others share the batched launches.
  std::vector<int> test, inner_b, inner_own;
  for (int k : inner) (B[k].c->L[0].ncell >= BATCH_OWN_CELLS ? inner_own : inner_b).push_back(k);
  for (int k : inner_own) {
    richards_ctx* c = B[k].c;
    BatchProgress& X = c->bp;
    run_cycle32(c);
    ++X.inner;
    ++X.k;
    if (c->opts.inner_rtol > 0.0 && X.k < c->opts.inner_cycles) {
      if (!fuse_defect(c)) {                   // (fused: the cycle left the defect norm in slot 1)
        BCK(cudaMemsetAsync(c->scratch + 1, 0, sizeof(unsigned long long), c->s));
        rich::residual32(view32(c, 0), phys<float>(c), c->soil.model, c->scratch + 1, c->s, c->tune_rbx[0]);
      }
      BCK(cudaMemcpyAsync(c->hscratch + 1, c->scratch + 1, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                          c->s));
    }
    own.push_back(k);
  }
  if (!inner_b.empty()) {
    TRY_B(bjoin(b, B, inner_b));
    batch_vcycle(b, B, inner_b, 0, true);
    for (int k : inner_b) {
      BatchProgress& X = B[k].c->bp;
      ++X.inner;
      ++X.k;
      if (B[k].c->opts.inner_rtol > 0.0 && X.k < B[k].c->opts.inner_cycles) test.push_back(k);
    }
    if (!test.empty()) {
      const size_t nb = sizeof(unsigned long long) * B.size();
      BCK(cudaMemsetAsync(b->dnorm, 0, nb, b->s));
      batch_stage(b, B, test, rich::BOP_RESID, 0, 0, true);
      BCK(cudaMemcpyAsync(b->hnorm, b->dnorm, nb, cudaMemcpyDeviceToHost, b->s));
    }
  }
  for (int k : own) BCK(cudaStreamSynchronize(B[k].c->s));
  if (!inner_b.empty()) BCK(cudaStreamSynchronize(b->s));
  // decisions
  std::vector<int> applied, applied_b;
  for (int k : inner) {
    richards_ctx* c = B[k].c;
    BatchProgress& X = c->bp;
    const bool alone = c->L[0].ncell >= BATCH_OWN_CELLS;
    bool end = X.k >= c->opts.inner_cycles;
    if (!end && c->opts.inner_rtol > 0.0) {
      const unsigned u = (unsigned)(alone ? c->hscratch[1] : b->hnorm[B[k].slot]);
      float f;
      std::memcpy(&f, &u, 4);
      end = (double)f <= X.rtol_in * X.rin0;
    }
    if (end) {
      applied.push_back(k);
      if (!alone) applied_b.push_back(k);
    }
  }
  if (!applied.empty()) {
    TRY_B(bfork(b, B, applied_b));
    for (int k : applied) {
      richards_ctx* c = B[k].c;
      rich::apply_delta(c->L[0].u, c->L[0].uf, c->L[0].ncell, c->s);
      ++c->bp.outer;
      c->bp.phase = BP_DEFECT;
    }
  }
  for (int k : defect) {
    richards_ctx* c = B[k].c;
    BatchProgress& X = c->bp;
    X.r = host_norm(c, 0, !X.use64) / c->a;
    if (!X.use64) {                            // a float-float defect: steer, or hand over to FP64
      const double prev = X.r_ff;
      X.r_ff = X.r;
      X.use64 = c->opts.precision == 2 && !std::isnan(X.r) &&
                (!(X.r > c->opts.tol) || X.outer >= c->opts.max_outer || X.r > 0.5 * prev);
      if (X.use64) continue;                   // the FP64 defect decides, next tick
    }
    if (X.outer == 0) X.r0 = X.r;
    if (!(X.r > c->opts.tol) || std::isnan(X.r)) { X.phase = BP_FINISH; continue; }
    if (X.outer >= c->opts.max_outer) { X.st = RICH_ENOCONV; X.phase = BP_FINISH; continue; }
    restrict_psi0(c);
    X.rin0 = X.r * c->a;
    X.rtol_in = std::max(c->opts.inner_rtol, 0.3 * c->opts.tol / X.r);
    if (c->opts.precision == 2 && X.rtol_in > c->opts.inner_rtol) X.use64 = true;
    if (top_defect_ready(c)) {
      const richards_status sd = defect_from_g(c);
      if (sd != RICH_OK) return bfail(b, sd, c->err);
    }
    X.k = 0;
    X.phase = BP_INNER;
  }
  for (int k : finish) {
    richards_ctx* c = B[k].c;
    BatchProgress& X = c->bp;
    richards_step_info& I = sinfo[k];
    I = richards_step_info{};
    I.cycles = X.inner;
    I.outer_iters = X.outer;
    I.scheme_used = c->scheme_used;
    I.resid0 = X.r0;
    I.resid = X.r;
    I.cell_updates = c->updates_host + (long long)c->hscratch[16];
    water_balance_done(c, X.r, X.fin == RICH_OK ? X.nbal : 0, &I);
    richards_status sk = X.fin;
    if (sk == RICH_OK)
      sk = std::isnan(X.r) ? fail(c, RICH_ENAN, "NaN in the iterate; state kept at psi^n") : finish_step_done(c, X.st);
    sst[k] = sk;
    done[k] = 1;
    X.phase = BP_IDLE;
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return bfail(b, RICH_ECUDA, std::string("batched launch: ") + cudaGetErrorString(e));
  return RICH_OK;
}

// Ticks until every context has done the steps it wants (until_all) or until
// one context that wanted steps has done all of them, or max_ticks ticks
// (> 0).  want: steps still wanted, counted down; steps[k], info[k]: steps
// completed here and their statistics (sums of cycles, outer iterations and
// updates; the rest from the last one); status[k]: the last step's.
richards_status batch_run(richards_batcher* b, std::vector<BatchCtx>& B, const double* dt, const int* scheme,
                          std::vector<int>& want, bool until_all, int max_ticks, std::vector<int>& steps,
                          std::vector<richards_status>& status, std::vector<richards_step_info>& info) {
  const int n = (int)B.size();
  std::vector<char> done(n, 0);
  std::vector<richards_status> sst(n, RICH_OK);
  std::vector<richards_step_info> sinfo(n);
  std::vector<int> all(n);
  for (int k = 0; k < n; ++k) all[k] = k;
  TRY_B(batch_upload(b, B, all));
  for (int tick = 0; max_ticks <= 0 || tick < max_ticks; ++tick) {
    bool busy = false;
    for (int k = 0; k < n; ++k) busy = busy || want[k] > 0 || B[k].c->bp.phase != BP_IDLE;
    if (!busy) break;
    TRY_B(batch_tick(b, B, dt, scheme, want, done, sst, sinfo));
    bool finished_one = false;
    for (int k = 0; k < n; ++k) {
      if (!done[k]) continue;
      richards_step_info& I = info[k];
      const richards_step_info& S = sinfo[k];
      if (steps[k] == 0) {
        I = S;
      } else {
        const int cyc = I.cycles + S.cycles, outer = I.outer_iters + S.outer_iters;
        const long long upd = I.cell_updates + S.cell_updates;
        const double r0 = I.resid0;
        I = S;
        I.cycles = cyc;
        I.outer_iters = outer;
        I.cell_updates = upd;
        I.resid0 = r0;
      }
      ++steps[k];
      status[k] = sst[k];
      want[k] = sst[k] == RICH_OK ? want[k] - 1 : 0;   // a failed step ends the context's run
      if (want[k] == 0) finished_one = true;
    }
    if (!until_all && finished_one) break;
  }
  return RICH_OK;
}

}  // namespace

// ==========================================================================
// extern "C" entry points
// ==========================================================================
extern "C" {

richards_status richards_create(const richards_grid* grid, const richards_opts* opts, void* stream,
                                richards_ctx** out) {
  if (!grid || !opts || !out) return RICH_EINVAL;
  *out = nullptr;
  if (grid->dim < 1 || grid->dim > 3) return RICH_EINVAL;
  for (int a = 0; a < 3; ++a) {
    if (grid->n[a] < 1) return RICH_EINVAL;
    if (a >= grid->dim && grid->n[a] != 1) return RICH_EINVAL;
    if (a < grid->dim && !(grid->L[a] > 0.0 && std::isfinite(grid->L[a]))) return RICH_EINVAL;
  }
  // launch grids put rows and planes on grid y/z (< 65536) and index a
  // level with 32-bit coordinates (< 2^31 cells)
  if (grid->n[1] > 65535 || grid->n[2] > 65535 ||
      (long long)grid->n[0] * grid->n[1] * grid->n[2] >= (1LL << 31))
    return RICH_EINVAL;
  const richards_opts& o = *opts;
  if (o.nu1 < 0 || o.nu2 < 0 || o.coarse_max_sweeps < 1 || o.max_cycles < 0 || o.coarsest_max_n < 1 ||
      !(o.tol > 0.0) || o.newton_iters < 0 || o.newton_iters > 200 || (o.kappa_mode != 0 && o.kappa_mode != 2) ||
      (o.ordering != 0 && o.ordering != 1) || (o.precision < 0 || o.precision > 2) || !(o.xi >= 0.0) || !(o.kappa >= 0.0) ||
      o.inner_cycles < 1 || o.max_outer < 0 || o.tail_cells < 0 || o.cycle_gamma < 1 || o.cycle_gamma > 3 ||
      o.gamma_levels < 0 || (o.graphs != 0 && o.graphs != 1) || (o.predictor != 0 && o.predictor != 1) ||
      o.fmg_cycles < 0 || o.fmg_cycles > 16 || (o.layout != 0 && o.layout != 1) || (o.bdf2_lag != 0 && o.bdf2_lag != 1) ||
      (o.sweep_planes != 1 && o.sweep_planes != 2 && o.sweep_planes != 4 && o.sweep_planes != 8))
    return RICH_EINVAL;
  richards_ctx* c = new richards_ctx();
  c->s = (cudaStream_t)stream;
  cudaGetDevice(&c->device);
  c->grid = *grid;
  c->opts = o;
  // hierarchy: halve every axis with n > 1 while max n > coarsest_max_n
  for (int a = 0; a < 3; ++a) {
    c->L[0].n[a] = grid->n[a];
    c->L[0].h[a] = a < grid->dim ? grid->L[a] / grid->n[a] : 1.0;
  }
  c->nlev = 1;
  for (;;) {
    const HLevel& F = c->L[c->nlev - 1];
    const int mx = std::max(F.n[0], std::max(F.n[1], F.n[2]));
    if (mx <= o.coarsest_max_n) break;
    if (o.max_levels > 0 && c->nlev >= o.max_levels) break;
    if (c->nlev >= MAXLEV) break;
    HLevel& C = c->L[c->nlev];
    for (int a = 0; a < 3; ++a) {
      C.n[a] = F.n[a] > 1 ? (F.n[a] + 1) / 2 : 1;
      C.h[a] = a < grid->dim ? grid->L[a] / C.n[a] : 1.0;
    }
    c->nlev++;
  }
  c->tail_start = c->nlev - 1;
  for (int l = 0; l < c->nlev; ++l)
    if ((long long)c->L[l].n[0] * c->L[l].n[1] * c->L[l].n[2] <= o.tail_cells) { c->tail_start = l; break; }
  const bool mixed = o.precision >= 1;
  c->coop_start = MAXLEV;
  if (o.precision >= 1 && COOP_CELLS > 0)
    for (int l = 1; l < c->tail_start; ++l)
      if ((long long)c->L[l].n[0] * c->L[l].n[1] * c->L[l].n[2] <= COOP_CELLS) { c->coop_start = l; break; }
  // the finest FP32 level of a big grid keeps its per-cell parameters in the
  // colour-split layout: a half-sweep then reads only its own colour's sectors
  // of them (the level must have an even n0 and lie above the coarse tail)
  if (mixed && o.layout == 0 && c->tail_start > 0 && grid->n[0] % 2 == 0 &&
      (long long)grid->n[0] * grid->n[1] * grid->n[2] >= (1LL << 20))
    c->L[0].cs = 1;
  richards_status st = RICH_OK;
  for (int l = 0; l < c->nlev && st == RICH_OK; ++l) {
    HLevel& H = c->L[l];
    H.ncell = (long long)H.n[0] * H.n[1] * H.n[2];
    const long long n = H.ncell;
    for (int f = 0; f < 6; ++f) H.nface[f] = (f / 2 < grid->dim) ? n / H.n[f / 2] : 0;
    double** d64[] = {&H.u, &H.ubar, &H.g, &H.d, &H.Kc};
    for (auto p : d64)
      if (st == RICH_OK) st = dalloc(c, p, n);
    for (int f = 0; f < 2 * grid->dim && st == RICH_OK; ++f) st = dalloc(c, &H.kb[f], H.nface[f]);
    if (mixed) {
      float** d32[] = {&H.uf, &H.ubarf, &H.gf, &H.df, &H.Kcf, &H.psi0f};
      for (auto p : d32)
        if (st == RICH_OK) st = dalloc(c, p, n);
      for (int f = 0; f < 2 * grid->dim && st == RICH_OK; ++f) st = dalloc(c, &H.kbf[f], H.nface[f]);
    }
  }
  const long long N = c->L[0].ncell;
  if (st == RICH_OK) st = dalloc(c, &c->psi_n, N);
  if (st == RICH_OK) st = dalloc(c, &c->psi_nm1, N);
  if (mixed) {
    if (st == RICH_OK) st = dalloc(c, &c->th_n, N);
    if (st == RICH_OK) st = dalloc(c, &c->th_nm1, N);
    if (st == RICH_OK) st = dalloc(c, &c->th_cur, N);
  }
  if (st == RICH_OK) st = dalloc(c, &c->dL64, c->nlev);
  if (st == RICH_OK) st = dalloc(c, &c->dX64, c->nlev);
  if (st == RICH_OK) st = dalloc(c, &c->dL32, c->nlev);
  if (st == RICH_OK) st = dalloc(c, &c->dX32, c->nlev);
  if (st == RICH_OK) st = dalloc(c, &c->scratch, NSCRATCH);
  if (st == RICH_OK) st = dalloc(c, &c->mass_part, MASS_PARTS + 1);
  if (st == RICH_OK && cudaMallocHost((void**)&c->hmass, (MASS_PARTS + 1) * sizeof(double)) != cudaSuccess)
    st = fail(c, RICH_ENOMEM, "cudaMallocHost failed");
  if (st == RICH_OK && cudaMallocHost((void**)&c->hscratch, NSCRATCH * sizeof(unsigned long long)) != cudaSuccess)
    st = fail(c, RICH_ENOMEM, "cudaMallocHost failed");
  if (st == RICH_OK && cudaMemsetAsync(c->scratch, 0, NSCRATCH * sizeof(unsigned long long), c->s) != cudaSuccess)
    st = fail(c, RICH_ECUDA, "cudaMemsetAsync failed");
  if (st != RICH_OK) {
    richards_destroy(c);
    return st;
  }
  *out = c;
  return RICH_OK;
}

void richards_destroy(richards_ctx* c) {
  if (!c) return;
  if (c->worker.joinable()) c->worker.join();
  if (c->s) cudaStreamSynchronize(c->s); else cudaDeviceSynchronize();
  graphs_reset(c);
  for (auto& r : c->prof_pending) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  for (void* p : c->allocs) cudaFree(p);
  for (void* p : c->bc_allocs) cudaFree(p);
  if (c->hscratch) cudaFreeHost(c->hscratch);
  if (c->hmass) cudaFreeHost(c->hmass);
  delete c;
}

const char* richards_last_error(const richards_ctx* c) { return c ? c->err.c_str() : "null context"; }

const char* richards_graph_status(const richards_ctx* c) {
  if (!c) return "null context";
  richards_ctx* m = const_cast<richards_ctx*>(c);
  m->graph_status.clear();
  if (!c->graph_err.empty()) m->graph_status = "cycle graph: " + c->graph_err;
  if (!c->loop_err.empty())
    m->graph_status += (m->graph_status.empty() ? "" : "; ") + std::string("inner-loop graph: ") + c->loop_err;
  return m->graph_status.c_str();
}

double richards_time(const richards_ctx* c) { return c ? c->t : 0.0; }
long long richards_ncell(const richards_ctx* c) { return c ? c->L[0].ncell : 0; }
int richards_nlevels(const richards_ctx* c) { return c ? c->nlev : 0; }

richards_status richards_level_dims(const richards_ctx* c, int level, int n_out[3]) {
  if (!c || !n_out || level < 0 || level >= c->nlev) return RICH_EINVAL;
  for (int a = 0; a < 3; ++a) n_out[a] = c->L[level].n[a];
  return RICH_OK;
}

richards_status richards_set_soil(richards_ctx* c, const richards_soil* s) {
  if (!c || !s) return RICH_EINVAL;
  if (c->busy.load()) return fail(c, RICH_EBUSY, "context busy: a batch is running on it");
  c->bp = BatchProgress{};
  cudaStreamSynchronize(c->s);
  graphs_reset(c);
  const long long N = c->L[0].ncell;
  if (const char* e = law_error(s->model, s->Ks, s->theta_s, s->theta_r, s->p1, s->p2, s->p3, s->p4,
                                s->p1_field != nullptr, s->p2_field != nullptr))
    return fail(c, RICH_EINVAL, e);
  if ((s->Ks_field && !finite_all(s->Ks_field, N)) || (s->p1_field && !finite_all(s->p1_field, N)) ||
      (s->p2_field && !finite_all(s->p2_field, N)))
    return fail(c, RICH_EINVAL, "non-finite value in a soil field");
  if (s->Ks_field)
    for (long long i = 0; i < N; ++i)
      if (!(s->Ks_field[i] > 0.0)) return fail(c, RICH_EINVAL, "Ks field must be positive");
  if (s->p2_field && s->model == RICH_VANGENUCHTEN)
    for (long long i = 0; i < N; ++i)
      if (!(s->p2_field[i] > 1.0)) return fail(c, RICH_EINVAL, "van Genuchten n field must exceed 1");
  c->soil = *s;
  c->soil.Ks_field = c->soil.p1_field = c->soil.p2_field = nullptr;
  c->layered = false;
  c->nmat = 0;
  c->th_n_valid = c->th_nm1_valid = false;   // cached theta belongs to the old soil
  c->het_Ks = s->Ks_field != nullptr;
  c->het_p1 = s->p1_field != nullptr;
  c->het_p2 = s->p2_field != nullptr;
  const bool mixed = c->opts.precision >= 1;
  if (c->het_Ks) {
    if (!c->Ks) TRY(dalloc(c, &c->Ks, N));
    CK(cudaMemcpyAsync(c->Ks, s->Ks_field, sizeof(double) * N, cudaMemcpyHostToDevice, c->s));
  }
  const double* fields[2] = {s->p1_field, s->p2_field};
  for (int k = 0; k < 2; ++k) {
    if (!fields[k]) continue;
    for (int l = 0; l < c->nlev; ++l) {
      HLevel& H = c->L[l];
      double*& p = k == 0 ? H.p1 : H.p2;
      float*& pf = k == 0 ? H.p1f : H.p2f;
      if (!p) TRY(dalloc(c, &p, H.ncell));
      if (mixed && !pf) TRY(dalloc(c, &pf, H.ncell));
    }
    CK(cudaMemcpyAsync(k == 0 ? c->L[0].p1 : c->L[0].p2, fields[k], sizeof(double) * N, cudaMemcpyHostToDevice,
                       c->s));
  }
  if (s->model == RICH_VANGENUCHTEN && c->het_p2) {   // m per cell for the FP64 laws: no division per evaluation
    if (!c->L[0].vgm) TRY(dalloc(c, &c->L[0].vgm, N));
    rich::vg_m_field(c->L[0].p2, c->L[0].vgm, N, c->s);
  }
  CK(cudaStreamSynchronize(c->s));
  c->soil_set = true;
  if (c->bc_set) {
    // coarse parameters need the transfer tables, built with the boundary conditions
    for (int l = 0; l + 1 < c->nlev; ++l) {
      const Level<double> F = view64(c, l), C = view64(c, l + 1);
      if (c->het_p1) rich::restrict64(F, C, xfer64(c, l), c->L[l].p1, nullptr, c->L[l + 1].p1, nullptr, c->s);
      if (c->het_p2) rich::restrict64(F, C, xfer64(c, l), c->L[l].p2, nullptr, c->L[l + 1].p2, nullptr, c->s);
    }
    if (mixed)
      for (int l = 0; l < c->nlev; ++l) {
        if (c->het_p1) to_float_at(c, l, c->L[l].p1, c->L[l].p1f);
        if (c->het_p2) to_float_at(c, l, c->L[l].p2, c->L[l].p2f);
      }
    TRY(check_launch(c));
    TRY(upload_views(c));
  }
  return RICH_OK;
}

richards_status richards_set_materials(richards_ctx* c, const richards_material* mats, int nmat,
                                       const unsigned char* index) {
  if (!c || !mats || !index) return RICH_EINVAL;
  if (c->busy.load()) return fail(c, RICH_EBUSY, "context busy: a batch is running on it");
  c->bp = BatchProgress{};
  if (nmat < 1 || nmat > rich::MAXMAT) return fail(c, RICH_EINVAL, "need 1 to 8 materials");
  for (int m = 0; m < nmat; ++m) {
    const richards_material& M = mats[m];
    if (const char* e = law_error(M.model, M.Ks, M.theta_s, M.theta_r, M.p1, M.p2, M.p3, M.p4, false, false))
      return fail(c, RICH_EINVAL, std::string("material ") + std::to_string(m) + ": " + e);
  }
  const long long N = c->L[0].ncell;
  for (long long i = 0; i < N; ++i)
    if (index[i] >= nmat) return fail(c, RICH_EINVAL, "material index out of range");
  cudaStreamSynchronize(c->s);
  graphs_reset(c);
  // material of every cell of every level: the fine index as given; a coarse
  // cell takes the material with the largest total restriction weight among
  // its fine cells (per-axis rows, weight (w0 w1) w2, summed over a2, a1, a0;
  // ties: the lower index)
  std::vector<std::vector<uint8_t>> mat(c->nlev);
  mat[0].assign(index, index + N);
  for (int l = 0; l + 1 < c->nlev; ++l) {
    const HLevel& F = c->L[l];
    const HLevel& C = c->L[l + 1];
    std::vector<Row> R[3];
    for (int a = 0; a < 3; ++a)
      if (!restriction_rows(F.n[a], C.n[a], R[a])) return fail(c, RICH_EINVAL, "restriction stencil too wide");
    mat[l + 1].resize(C.ncell);
    for (int J2 = 0; J2 < C.n[2]; ++J2)
      for (int J1 = 0; J1 < C.n[1]; ++J1)
        for (int J0 = 0; J0 < C.n[0]; ++J0) {
          const Row &r0 = R[0][J0], &r1 = R[1][J1], &r2 = R[2][J2];
          double w[rich::MAXMAT] = {0.0};
          for (int a2 = 0; a2 < r2.cnt; ++a2)
            for (int a1 = 0; a1 < r1.cnt; ++a1)
              for (int a0 = 0; a0 < r0.cnt; ++a0) {
                const long long i = r0.idx[a0] + (long long)F.n[0] * (r1.idx[a1] + (long long)F.n[1] * r2.idx[a2]);
                w[mat[l][i]] += r0.w[a0] * r1.w[a1] * r2.w[a2];
              }
          int best = 0;
          for (int m = 1; m < nmat; ++m)
            if (w[m] > w[best]) best = m;
          mat[l + 1][J0 + (long long)C.n[0] * (J1 + (long long)C.n[1] * J2)] = (uint8_t)best;
        }
  }
  // per-level arrays: material index, and p1, p2 (and the fine Ks) of each
  // cell's material, not restricted
  const bool mixed = c->opts.precision >= 1;
  if (!c->Ks) TRY(dalloc(c, &c->Ks, N));
  std::vector<double> hKs(N);
  for (long long i = 0; i < N; ++i) hKs[i] = mats[index[i]].Ks;
  CK(cudaMemcpyAsync(c->Ks, hKs.data(), sizeof(double) * N, cudaMemcpyHostToDevice, c->s));
  std::vector<std::vector<double>> hp(2 * c->nlev);
  for (int l = 0; l < c->nlev; ++l) {
    HLevel& H = c->L[l];
    if (!H.mat) TRY(dalloc(c, &H.mat, H.ncell));
    if (!H.p1) TRY(dalloc(c, &H.p1, H.ncell));
    if (!H.p2) TRY(dalloc(c, &H.p2, H.ncell));
    if (mixed && !H.p1f) TRY(dalloc(c, &H.p1f, H.ncell));
    if (mixed && !H.p2f) TRY(dalloc(c, &H.p2f, H.ncell));
    std::vector<double>& q1 = hp[2 * l];
    std::vector<double>& q2 = hp[2 * l + 1];
    q1.resize(H.ncell);
    q2.resize(H.ncell);
    for (long long i = 0; i < H.ncell; ++i) {
      q1[i] = mats[mat[l][i]].p1;
      q2[i] = mats[mat[l][i]].p2;
    }
    CK(cudaMemcpyAsync(H.mat, mat[l].data(), H.ncell, cudaMemcpyHostToDevice, c->s));
    CK(cudaMemcpyAsync(H.p1, q1.data(), sizeof(double) * H.ncell, cudaMemcpyHostToDevice, c->s));
    CK(cudaMemcpyAsync(H.p2, q2.data(), sizeof(double) * H.ncell, cudaMemcpyHostToDevice, c->s));
    if (mixed) {
      to_float_at(c, l, H.p1, H.p1f);
      to_float_at(c, l, H.p2, H.p2f);
    }
  }
  // material tables (FP64, FP32, float-float)
  if (!c->dmat64) TRY(dalloc(c, &c->dmat64, rich::MAXMAT));
  if (!c->dmat32) TRY(dalloc(c, &c->dmat32, rich::MAXMAT));
  if (!c->dmatdd) TRY(dalloc(c, &c->dmatdd, rich::MAXMAT));
  rich::MatLaw<double> t64[rich::MAXMAT] = {};
  rich::MatLaw<float> t32[rich::MAXMAT] = {};
  rich::DDMat tdd[rich::MAXMAT] = {};
  for (int m = 0; m < nmat; ++m) {
    const richards_material& M = mats[m];
    t64[m] = rich::MatLaw<double>{M.model, M.theta_s, M.theta_r, M.p3, M.p4};
    t32[m] = rich::MatLaw<float>{M.model, (float)M.theta_s, (float)M.theta_r, (float)M.p3, (float)M.p4};
    tdd[m] = rich::make_ddmat(t64[m]);
  }
  CK(cudaMemcpyAsync(c->dmat64, t64, sizeof(t64), cudaMemcpyHostToDevice, c->s));
  CK(cudaMemcpyAsync(c->dmat32, t32, sizeof(t32), cudaMemcpyHostToDevice, c->s));
  CK(cudaMemcpyAsync(c->dmatdd, tdd, sizeof(tdd), cudaMemcpyHostToDevice, c->s));
  TRY(check_launch(c));
  CK(cudaStreamSynchronize(c->s));
  c->nmat = nmat;
  for (int m = 0; m < nmat; ++m) c->mats[m] = mats[m];
  richards_soil s0{};
  s0.model = rich::COMPOSITE;
  s0.Ks = mats[0].Ks;
  s0.theta_s = mats[0].theta_s;
  s0.theta_r = mats[0].theta_r;
  s0.p1 = mats[0].p1; s0.p2 = mats[0].p2; s0.p3 = mats[0].p3; s0.p4 = mats[0].p4;
  c->soil = s0;
  c->layered = true;
  c->het_Ks = c->het_p1 = c->het_p2 = true;
  c->th_n_valid = c->th_nm1_valid = false;
  c->soil_set = true;
  return upload_views(c);
}

static richards_status refresh_sink(richards_ctx* c) {
  if (!c->sink.enabled || !c->bc_set) return RICH_OK;
  const bool mixed = c->opts.precision >= 1;
  for (int l = 0; l < c->nlev; ++l) {
    HLevel& H = c->L[l];
    if (!H.smax) TRY(dalloc(c, &H.smax, H.ncell));
    if (mixed && !H.smaxf) TRY(dalloc(c, &H.smaxf, H.ncell));
  }
  rich::sink_coef(geom(c, 0), c->sink.Tp, c->sink.root_depth, c->sink.root_decay, c->L[0].smax, c->s);
  for (int l = 0; l + 1 < c->nlev; ++l)
    rich::restrict64(view64(c, l), view64(c, l + 1), xfer64(c, l), c->L[l].smax, nullptr, c->L[l + 1].smax, nullptr,
                     c->s);
  if (mixed)
    for (int l = 0; l < c->nlev; ++l) to_float_at(c, l, c->L[l].smax, c->L[l].smaxf);
  TRY(check_launch(c));
  return upload_views(c);
}

richards_status richards_set_sink(richards_ctx* c, const richards_sink* k) {
  if (!c || !k) return RICH_EINVAL;
  if (c->busy.load()) return fail(c, RICH_EBUSY, "context busy: a batch is running on it");
  c->bp = BatchProgress{};
  cudaStreamSynchronize(c->s);
  graphs_reset(c);
  if (const char* e = rich::sink_error(*k)) return fail(c, RICH_EINVAL, e);
  c->sink = *k;
  return refresh_sink(c);
}

richards_status richards_set_bc(richards_ctx* c, const richards_bc* b) {
  if (!c || !b) return RICH_EINVAL;
  if (c->busy.load()) return fail(c, RICH_EBUSY, "context busy: a batch is running on it");
  c->bp = BatchProgress{};
  cudaStreamSynchronize(c->s);
  graphs_reset(c);
  const int dim = c->grid.dim;
  const HLevel& F = c->L[0];
  if (const char* e = rich::bc_error(*b, dim)) return fail(c, RICH_EINVAL, e);
  for (int f = 0; f < 2 * dim; ++f)
    if (b->value_field[f] && !finite_all(b->value_field[f], F.nface[f]))
      return fail(c, RICH_EINVAL, "non-finite boundary field");
  // release tables and fields of an earlier call
  cudaStreamSynchronize(c->s);
  for (void* p : c->bc_allocs) cudaFree(p);
  c->bc_allocs.clear();
  c->bc = *b;
  rich::BcDev bd{};
  for (int f = 0; f < 6; ++f) {
    bd.kind[f] = f < 2 * dim ? b->kind[f] : RICH_BC_NOFLUX;
    bd.value[f] = f < 2 * dim ? b->value[f] : 0.0;
    bd.vfield[f] = nullptr;
    bd.mask[f] = nullptr;
    c->bc.value_field[f] = nullptr;
    c->bc.mask_field[f] = nullptr;
    if (f >= 2 * dim) continue;
    if (b->value_field[f]) {
      double* p;
      TRY(dalloc(c, &p, F.nface[f], &c->bc_allocs));
      CK(cudaMemcpy(p, b->value_field[f], sizeof(double) * F.nface[f], cudaMemcpyHostToDevice));
      bd.vfield[f] = p;
    }
    if (b->mask_field[f]) {
      unsigned char* p;
      TRY(dalloc(c, &p, F.nface[f], &c->bc_allocs));
      CK(cudaMemcpy(p, b->mask_field[f], F.nface[f], cudaMemcpyHostToDevice));
      bd.mask[f] = p;
    }
  }
  c->bcdev = bd;
  for (int l = 0; l + 1 < c->nlev; ++l)
    for (int ax = 0; ax < 3; ++ax) {
      double slo = 1.0, shi = 1.0;
      if (ax < dim) {
        if (b->kind[2 * ax] == RICH_BC_DIRICHLET && !b->mask_field[2 * ax]) slo = -1.0;
        if (b->kind[2 * ax + 1] == RICH_BC_DIRICHLET && !b->mask_field[2 * ax + 1]) shi = -1.0;
      }
      TRY(build_axis_tables(c, l, ax, slo, shi));
    }
  c->bc_set = true;
  TRY(upload_views(c));
  if (c->soil_set && !c->layered) {
    // re-run the coarse parameter restriction with the new tables (a
    // layered soil's coarse parameters come from the coarse materials)
    for (int l = 0; l + 1 < c->nlev; ++l) {
      const Level<double> Fv = view64(c, l), Cv = view64(c, l + 1);
      if (c->het_p1) rich::restrict64(Fv, Cv, xfer64(c, l), c->L[l].p1, nullptr, c->L[l + 1].p1, nullptr, c->s);
      if (c->het_p2) rich::restrict64(Fv, Cv, xfer64(c, l), c->L[l].p2, nullptr, c->L[l + 1].p2, nullptr, c->s);
    }
    if (c->opts.precision >= 1)
      for (int l = 0; l < c->nlev; ++l) {
        if (c->het_p1) to_float_at(c, l, c->L[l].p1, c->L[l].p1f);
        if (c->het_p2) to_float_at(c, l, c->L[l].p2, c->L[l].p2f);
      }
    TRY(check_launch(c));
  }
  return refresh_sink(c);
}

richards_status richards_set_state(richards_ctx* c, const double* psi, const double* psi_prev, double t) {
  if (!c || !psi) return RICH_EINVAL;
  if (c->busy.load()) return fail(c, RICH_EBUSY, "context busy: a batch is running on it");
  c->bp = BatchProgress{};
  const long long N = c->L[0].ncell;
  if (!std::isfinite(t)) return fail(c, RICH_EINVAL, "non-finite time");
  // the values are staged in two finest-level work arrays (FAS restricted
  // iterate and defect, rewritten by every step) and checked there on the
  // device, so that a rejected state leaves the context as it was.  The same
  // pass compares them with the context's own psi^n and psi^{n-1} where those
  // have a theta cache: a state handed back bit for bit keeps its cache
  // (flag bit 1: psi^n changed, bit 2: psi^{n-1} changed)
  HLevel& F = c->L[0];
  const bool cmp_n = c->have_state && c->th_n_valid;
  const bool cmp_nm1 = psi_prev && c->have_state && c->have_prev && c->th_nm1_valid;
  CK(cudaMemcpyAsync(F.ubar, psi, sizeof(double) * N, cudaMemcpyHostToDevice, c->s));
  if (psi_prev) CK(cudaMemcpyAsync(F.d, psi_prev, sizeof(double) * N, cudaMemcpyHostToDevice, c->s));
  unsigned* flags = (unsigned*)(c->scratch + 17);
  CK(cudaMemsetAsync(flags, 0, sizeof(unsigned), c->s));
  rich::screen_state(F.ubar, cmp_n ? c->psi_n : nullptr, N, 2u, flags, c->s);
  if (psi_prev) rich::screen_state(F.d, cmp_nm1 ? c->psi_nm1 : nullptr, N, 4u, flags, c->s);
  TRY(check_launch(c));
  CK(cudaMemcpyAsync(c->hscratch + 17, c->scratch + 17, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->s));
  CK(cudaStreamSynchronize(c->s));
  const unsigned fl = (unsigned)c->hscratch[17];
  if (fl & 1u) return fail(c, RICH_EINVAL, "non-finite state");
  const bool same_n = cmp_n && !(fl & 2u), same_nm1 = cmp_nm1 && !(fl & 4u);
  if (!same_n) CK(cudaMemcpyAsync(c->psi_n, F.ubar, sizeof(double) * N, cudaMemcpyDeviceToDevice, c->s));
  if (psi_prev && !same_nm1)
    CK(cudaMemcpyAsync(c->psi_nm1, F.d, sizeof(double) * N, cudaMemcpyDeviceToDevice, c->s));
  CK(cudaStreamSynchronize(c->s));
  c->have_state = true;
  c->have_prev = psi_prev != nullptr;
  c->th_n_valid = same_n;
  c->th_nm1_valid = same_nm1;
  c->t = t;
  return RICH_OK;
}

richards_status richards_get_state(richards_ctx* c, double* out, int on_device) {
  if (!c || !out) return RICH_EINVAL;
  if (c->busy.load()) return fail(c, RICH_EBUSY, "context busy: a batch is running on it");
  if (!c->have_state) return fail(c, RICH_EINVAL, "state not set");
  CK(cudaMemcpyAsync(out, c->psi_n, sizeof(double) * c->L[0].ncell,
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->s));
  CK(cudaStreamSynchronize(c->s));
  return RICH_OK;
}

richards_status richards_soil_eval(richards_ctx* c, const double* psi, double* theta, double* K, int arith,
                                   int on_device) {
  if (!c || !psi || (arith != 0 && arith != 1)) return RICH_EINVAL;
  if (c->busy.load()) return fail(c, RICH_EBUSY, "context busy: a batch is running on it");
  if (!c->soil_set) return fail(c, RICH_EINVAL, "soil not set");
  const long long n = c->L[0].ncell;
  const size_t bytes = sizeof(double) * n;
  const double* dpsi = psi;
  double *dth = theta, *dK = K, *tmp = nullptr;
  if (!on_device) {
    CK(cudaMallocAsync((void**)&tmp, 3 * bytes, c->s));
    CK(cudaMemcpyAsync(tmp, psi, bytes, cudaMemcpyHostToDevice, c->s));
    dpsi = tmp;
    dth = theta ? tmp + n : nullptr;
    dK = K ? tmp + 2 * n : nullptr;
  }
  HLevel& F = c->L[0];
  const Phys<double> P = phys<double>(c);
  rich::soil_eval(n, dpsi, c->het_Ks ? c->Ks : nullptr, c->soil.Ks, c->het_p1 ? F.p1 : nullptr,
                  c->het_p2 ? F.p2 : nullptr, fine_mat(c), P, rich::make_ddphys(P), c->soil.model, arith == 1, dth,
                  dK, c->s);
  richards_status st = check_launch(c);
  if (!on_device) {
    if (st == RICH_OK && theta) st = cudaMemcpyAsync(theta, dth, bytes, cudaMemcpyDeviceToHost, c->s) == cudaSuccess
                                         ? RICH_OK : fail(c, RICH_ECUDA, "cudaMemcpyAsync failed");
    if (st == RICH_OK && K) st = cudaMemcpyAsync(K, dK, bytes, cudaMemcpyDeviceToHost, c->s) == cudaSuccess
                                     ? RICH_OK : fail(c, RICH_ECUDA, "cudaMemcpyAsync failed");
    cudaFreeAsync(tmp, c->s);
  }
  CK(cudaStreamSynchronize(c->s));
  return st;
}

richards_status richards_prepare(richards_ctx* c, double dt, int scheme, int* scheme_used) {
  if (!c) return RICH_EINVAL;
  if (c->busy.load()) return fail(c, RICH_EBUSY, "context busy: a batch is running on it");
  TRY(do_prepare(c, dt, scheme));
  if (scheme_used) *scheme_used = c->scheme_used;
  CK(cudaStreamSynchronize(c->s));
  return RICH_OK;
}

static richards_status step_impl(richards_ctx* c, double dt, int scheme, richards_step_info* info);

richards_status richards_step(richards_ctx* c, double dt, int scheme, richards_step_info* info) {
  if (!c) return RICH_EINVAL;
  if (c->busy.load()) return fail(c, RICH_EBUSY, "context busy: a batch is running on it");
  return step_impl(c, dt, scheme, info);
}

// A grid of at most RICHARDS_NOALLOC_MAX_CELLS cells in FP64 (no FMG start):
// the step -- preparation, stop tests and every cycle -- runs in one thread
// block on the context's own hierarchy, one launch and one synchronisation
// instead of a launch per stage and a host round trip per cycle (the same
// arithmetic as the grid path: apply_N, the point update and the transfers
// are shared; layered soils included).
static bool small_path(const richards_ctx* c) {
  return c->opts.precision == 0 && c->opts.fmg_cycles == 0 && c->L[0].ncell <= RICHARDS_NOALLOC_MAX_CELLS &&
         c->prof == 0;
}

static richards_status step_small(richards_ctx* c, double dt, int scheme, richards_step_info* info) {
  if (!c->soil_set) return fail(c, RICH_EINVAL, "soil not set");
  if (!c->bc_set) return fail(c, RICH_EINVAL, "boundary conditions not set");
  if (!c->have_state) return fail(c, RICH_EINVAL, "state not set");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, RICH_EINVAL, "dt must be positive and finite");
  if (scheme != 1 && scheme != 2) return fail(c, RICH_EINVAL, "scheme must be 1 (BDF1) or 2 (BDF2)");
  if (scheme == 2 && !c->have_prev) scheme = 1;
  c->scheme_used = scheme;
  c->dt = dt;
  c->a = scheme == 1 ? 1.0 / dt : 1.5 / dt;
  c->prepared = false;          // the coarse levels of the grid path are not set up by this step
  HLevel& F = c->L[0];
  richards_soil soil = c->soil;
  soil.Ks_field = c->het_Ks ? c->Ks : nullptr;
  soil.p1_field = c->het_p1 ? F.p1 : nullptr;
  soil.p2_field = c->het_p2 ? F.p2 : nullptr;
  richards_bc bc = c->bc;
  for (int f = 0; f < 6; ++f) {
    bc.value_field[f] = c->bcdev.vfield[f];
    bc.mask_field[f] = c->bcdev.mask[f];
  }
  std::vector<Level<double>> lv(c->nlev);
  std::vector<Xfer<double>> xv(c->nlev);
  for (int l = 0; l < c->nlev; ++l) {
    lv[l] = view64(c, l);
    xv[l] = xfer64(c, l);
  }
  const rich::SmallCtx cx{c->nlev, lv.data(), xv.data(), c->layered ? c->dmat64 : nullptr};
  double* stats = (double*)(c->hscratch + 32);         // 5 doubles of the pinned host slots
  if (rich::small_step(&c->grid, &soil, &bc, &c->sink, &c->opts, dt, scheme, c->psi_n,
                       scheme == 2 ? c->psi_nm1 : nullptr, F.u, (double*)(c->scratch + 32), &cx, c->opts.ordering,
                       stats, c->s) != RICH_OK)
    return fail(c, RICH_ECUDA, "single-block step failed");
  const double r = stats[2];
  const richards_status st = (richards_status)(int)stats[3];
  if (info) {
    info->cycles = (int)stats[0];
    info->outer_iters = 0;
    info->scheme_used = scheme;
    info->resid0 = stats[1];
    info->resid = r;
    info->cell_updates = (long long)stats[4];
  }
  TRY(water_balance(c, r, info, nullptr, nullptr, nullptr));
  return finish_step(c, r, st == RICH_OK ? RICH_OK : RICH_ENOCONV);
}

static richards_status step_impl(richards_ctx* c, double dt, int scheme, richards_step_info* info) {
  if (small_path(c)) return step_small(c, dt, scheme, info);
  c->updates_host = 0;
  CK(cudaMemsetAsync(c->scratch + 16, 0, sizeof(unsigned long long), c->s));
  TRY(do_prepare(c, dt, scheme));
  return c->opts.precision >= 1 ? step_mixed(c, info) : step_fp64(c, info);
}

static richards_status solve_impl(richards_ctx* c, double dt, int nsteps, int scheme, richards_step_info* last) {
  for (int k = 0; k < nsteps; ++k) TRY(step_impl(c, dt, scheme, last));
  return RICH_OK;
}

richards_status richards_solve(richards_ctx* c, double dt, int nsteps, int scheme, richards_step_info* last) {
  if (!c || nsteps < 0) return RICH_EINVAL;
  if (c->busy.load()) return fail(c, RICH_EBUSY, "context busy: a batch is running on it");
  return solve_impl(c, dt, nsteps, scheme, last);
}

richards_status richards_batch_submit(richards_ctx* const* ctxs, int n, double dt, int nsteps, int scheme) {
  if (!ctxs || n < 0 || nsteps < 0 || !(dt > 0.0) || (scheme != 1 && scheme != 2)) return RICH_EINVAL;
  for (int k = 0; k < n; ++k) {
    if (!ctxs[k]) return RICH_EINVAL;
    if (ctxs[k]->busy.load()) return RICH_EBUSY;
    for (int j = 0; j < k; ++j)
      if (ctxs[j] == ctxs[k]) return RICH_EINVAL;
  }
  for (int k = 0; k < n; ++k) {
    richards_ctx* c = ctxs[k];
    if (c->worker.joinable()) c->worker.join();
    c->busy.store(1);
    c->batch_info = richards_step_info{};
    c->worker = std::thread([c, dt, nsteps, scheme]() {
      cudaSetDevice(c->device);
      richards_step_info acc{}, last{};
      richards_status st = RICH_OK;
      for (int k = 0; k < nsteps && st == RICH_OK; ++k) {
        st = step_impl(c, dt, scheme, &last);
        acc.cycles += last.cycles;
        acc.outer_iters += last.outer_iters;
        acc.cell_updates += last.cell_updates;
        acc.scheme_used = last.scheme_used;
        acc.resid = last.resid;
        acc.mass_defect = last.mass_defect;
        acc.err_bound = last.err_bound;
        if (k == 0) acc.resid0 = last.resid0;
      }
      c->batch_info = acc;
      c->batch_status = st;
      c->busy.store(0);
    });
  }
  return RICH_OK;
}

richards_status richards_batch_poll(richards_ctx* const* ctxs, int n, int* done, richards_status* status,
                                    richards_step_info* info) {
  if (!ctxs || n < 0 || !done) return RICH_EINVAL;
  for (int k = 0; k < n; ++k) {
    richards_ctx* c = ctxs[k];
    if (!c) return RICH_EINVAL;
    done[k] = c->busy.load() ? 0 : 1;
    if (done[k]) {
      if (c->worker.joinable()) c->worker.join();
      if (status) status[k] = c->batch_status;
      if (info) info[k] = c->batch_info;
    }
  }
  return RICH_OK;
}

richards_status richards_math_eval(int fn, const double* x, double* y, long long n, void* stream) {
  if (fn < 0 || fn > 7 || n < 0 || (n > 0 && (!x || !y))) return RICH_EINVAL;
  if (n == 0) return RICH_OK;
  rich::math_eval(fn, x, y, n, (cudaStream_t)stream);
  if (cudaGetLastError() != cudaSuccess) return RICH_ECUDA;
  return cudaStreamSynchronize((cudaStream_t)stream) == cudaSuccess ? RICH_OK : RICH_ECUDA;
}

richards_status richards_set_coop(richards_ctx* c, long long max_cells) {
  if (!c || max_cells < 0) return RICH_EINVAL;
  if (c->busy.load()) return fail(c, RICH_EBUSY, "context busy: a batch is running on it");
  cudaStreamSynchronize(c->s);
  graphs_reset(c);
  c->coop_start = MAXLEV;
  c->coop_blocks = 0;
  if (max_cells > 0 && c->opts.precision >= 1)
    for (int l = 1; l < c->tail_start; ++l)
      if (c->L[l].ncell <= max_cells) { c->coop_start = l; break; }
  return RICH_OK;
}

richards_status richards_set_launch(richards_ctx* c, int level, int planes, int block_x, int resid_block_x) {
  if (!c || level < 0 || level >= c->nlev) return RICH_EINVAL;
  if (c->busy.load()) return fail(c, RICH_EBUSY, "context busy: a batch is running on it");
  auto bx_ok = [](int b) { return b == 0 || b == 32 || b == 64 || b == 128 || b == 256; };
  if (!(planes == 0 || planes == 1 || planes == 2 || planes == 4 || planes == 8) || !bx_ok(block_x) ||
      !bx_ok(resid_block_x) || (planes > 1 && block_x > 128))
    return fail(c, RICH_EINVAL, "planes in {0,1,2,4,8}, block sizes in {0,32,64,128,256} (128 at most with planes > 1)");
  if (level == 0 && planes > 0 && fuse_defect(c) && planes != 2)
    return fail(c, RICH_EINVAL, "the finest level's defect-writing half-sweep needs two planes");
  cudaStreamSynchronize(c->s);
  graphs_reset(c);
  c->tune_planes[level] = planes;
  c->tune_bx[level] = block_x;
  c->tune_rbx[level] = resid_block_x;
  return RICH_OK;
}

richards_status richards_autotune(richards_ctx* c, int reps, int* planes_out, int* bx_out, int* rbx_out) {
  if (!c || reps < 1 || reps > 100) return RICH_EINVAL;
  if (c->busy.load()) return fail(c, RICH_EBUSY, "context busy: a batch is running on it");
  if (!c->prepared || c->opts.precision < 1 || c->opts.ordering != 1)
    return fail(c, RICH_EINVAL, "autotune needs a prepared mixed-mode context with red-black sweeps");
  cudaStreamSynchronize(c->s);
  graphs_reset(c);
  const Phys<float> P = phys<float>(c);
  const int model = c->soil.model;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  richards_status st = RICH_OK;
  for (int l = 0; l < c->tail_start && st == RICH_OK; ++l) {
    HLevel& H = c->L[l];
    if (H.ncell < (1LL << 15)) continue;        // small levels: bound by their own latency
    const Level<float> F = view32(c, l);
    float* save = nullptr;
    if (cudaMallocAsync((void**)&save, sizeof(float) * 2 * H.ncell, c->s) != cudaSuccess) {
      st = fail(c, RICH_ENOMEM, "autotune: no room for the saved state");
      break;
    }
    cudaMemcpyAsync(save, H.uf, sizeof(float) * H.ncell, cudaMemcpyDeviceToDevice, c->s);
    cudaMemcpyAsync(save + H.ncell, H.df, sizeof(float) * H.ncell, cudaMemcpyDeviceToDevice, c->s);
    // every candidate computes the same values (one cell's arithmetic does
    // not depend on the launch shape); each starts from the saved state
    auto time_it = [&](auto&& launch) -> float {
      launch();                                 // warm-up
      cudaEventRecord(e0, c->s);
      for (int r = 0; r < reps; ++r) launch();
      cudaEventRecord(e1, c->s);
      cudaEventSynchronize(e1);
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      cudaMemcpyAsync(H.uf, save, sizeof(float) * H.ncell, cudaMemcpyDeviceToDevice, c->s);
      return ms;
    };
    const bool fixed2 = l == 0 && fuse_defect(c);
    const int plist[4] = {1, 2, 4, 8}, blist[4] = {32, 64, 128, 256};
    float best = INFINITY;
    int bp = 0, bb = 0;
    for (int pl : plist) {
      if (fixed2 && pl != 2) continue;
      if (pl > 1 && (F.dim < 3 || F.n2 < 2 * pl)) continue;
      for (int bx : blist) {
        if (pl > 1 && bx > 128) continue;
        const float ms = time_it([&] {
          rich::sweep32(F, P, model, 0, pl, c->s, bx);
          rich::sweep32(F, P, model, 1, pl, c->s, bx);
        });
        if (ms < best) { best = ms; bp = pl; bb = bx; }
      }
    }
    float bestr = INFINITY;
    int br = 0;
    for (int bx : blist) {
      const float ms = time_it([&] { rich::residual32(F, P, model, nullptr, c->s, bx); });
      if (ms < bestr) { bestr = ms; br = bx; }
    }
    c->tune_planes[l] = bp;
    c->tune_bx[l] = bb;
    c->tune_rbx[l] = br;
    cudaMemcpyAsync(H.df, save + H.ncell, sizeof(float) * H.ncell, cudaMemcpyDeviceToDevice, c->s);
    cudaFreeAsync(save, c->s);
    if (cudaGetLastError() != cudaSuccess) st = fail(c, RICH_ECUDA, "autotune: a candidate launch failed");
  }
  cudaStreamSynchronize(c->s);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (int l = 0; l < c->nlev; ++l) {
    if (planes_out) planes_out[l] = planes_at(c, l);
    if (bx_out) bx_out[l] = c->tune_bx[l];
    if (rbx_out) rbx_out[l] = c->tune_rbx[l];
  }
  return st;
}

richards_status richards_batcher_create(void* stream, int max_contexts, richards_batcher** out) {
  if (!out || max_contexts < 1 || max_contexts > 4096) return RICH_EINVAL;
  *out = nullptr;
  richards_batcher* b = new richards_batcher();
  b->s = (cudaStream_t)stream;
  b->cap = max_contexts;
  const size_t bytes = sizeof(rich::BJob32) * (size_t)max_contexts * MAXLEV;
  const size_t nbytes = sizeof(unsigned long long) * (size_t)max_contexts;
  b->join.assign(max_contexts, nullptr);
  bool ok = cudaMalloc((void**)&b->dtable, bytes) == cudaSuccess &&
            cudaMallocHost((void**)&b->htable, bytes) == cudaSuccess &&
            cudaMalloc((void**)&b->dnorm, nbytes) == cudaSuccess &&
            cudaMallocHost((void**)&b->hnorm, nbytes) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
  for (int k = 0; ok && k < max_contexts; ++k)
    ok = cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    richards_batcher_destroy(b);
    return RICH_ENOMEM;
  }
  *out = b;
  return RICH_OK;
}

void richards_batcher_destroy(richards_batcher* b) {
  if (!b) return;
  if (b->s) cudaStreamSynchronize(b->s); else cudaDeviceSynchronize();
  if (b->dtable) cudaFree(b->dtable);
  if (b->htable) cudaFreeHost(b->htable);
  if (b->dnorm) cudaFree(b->dnorm);
  if (b->hnorm) cudaFreeHost(b->hnorm);
  if (b->fork) cudaEventDestroy(b->fork);
  for (cudaEvent_t e : b->join)
    if (e) cudaEventDestroy(e);
  delete b;
}

const char* richards_batcher_last_error(const richards_batcher* b) { return b ? b->err.c_str() : "null batcher"; }

}  // extern "C"

namespace {

// checks shared by richards_batcher_step and _advance
richards_status batch_check(richards_batcher* b, richards_ctx* const* ctxs, int n, const double* dt,
                            const int* scheme) {
  if (n > b->cap) return bfail(b, RICH_EINVAL, "more contexts than the batcher holds");
  const richards_opts* o0 = ctxs[0] ? &ctxs[0]->opts : nullptr;
  for (int k = 0; k < n; ++k) {
    const richards_ctx* c = ctxs[k];
    if (!c || !o0) return bfail(b, RICH_EINVAL, "null context");
    for (int q = 0; q < k; ++q)
      if (ctxs[q] == c) return bfail(b, RICH_EINVAL, "a context appears twice");
    if (c->busy.load()) return bfail(b, RICH_EBUSY, "context busy: a batch is running on it");
    const richards_opts& o = c->opts;
    if (o.precision < 1 || o.ordering != 1 || o.fmg_cycles != 0)
      return bfail(b, RICH_EINVAL, "batched steps need mixed precision, red-black sweeps and no FMG start");
    if (o.nu1 != o0->nu1 || o.nu2 != o0->nu2 || o.cycle_gamma != o0->cycle_gamma ||
        o.gamma_levels != o0->gamma_levels || o.coarse_max_sweeps != o0->coarse_max_sweeps ||
        o.coarse_rtol != o0->coarse_rtol || o.inner_cycles != o0->inner_cycles)
      return bfail(b, RICH_EINVAL, "batched contexts must share the cycle options");
    if (!(dt[k] > 0.0) || !std::isfinite(dt[k]) || (scheme[k] != 1 && scheme[k] != 2))
      return bfail(b, RICH_EINVAL, "bad dt or scheme");
  }
  return RICH_OK;
}

richards_status batch_call(richards_batcher* b, richards_ctx* const* ctxs, int n, const double* dt,
                           const int* scheme, std::vector<int>& want, bool until_all, int max_ticks,
                           std::vector<int>& steps, std::vector<richards_status>& status,
                           std::vector<richards_step_info>& info) {
  std::vector<BatchCtx> B(n);
  for (int k = 0; k < n; ++k) {
    B[k].c = ctxs[k];
    B[k].slot = k;
    ctxs[k]->busy.store(1);
  }
  const richards_status st = batch_run(b, B, dt, scheme, want, until_all, max_ticks, steps, status, info);
  for (int k = 0; k < n; ++k) {
    if (st != RICH_OK) ctxs[k]->bp = BatchProgress{};     // a failed call leaves no step in progress
    ctxs[k]->busy.store(0);
  }
  return st;
}

}  // namespace

extern "C" {

richards_status richards_batcher_step(richards_batcher* b, richards_ctx* const* ctxs, int n, const double* dt,
                                      const int* scheme, richards_status* status, richards_step_info* info) {
  if (!b || !ctxs || !dt || !scheme || n < 1) return RICH_EINVAL;
  TRY_B(batch_check(b, ctxs, n, dt, scheme));
  std::vector<int> want(n, 1), steps(n, 0);
  std::vector<richards_status> sst(n, RICH_OK);
  std::vector<richards_step_info> inf(n);
  const richards_status st = batch_call(b, ctxs, n, dt, scheme, want, true, 0, steps, sst, inf);
  for (int k = 0; k < n; ++k) {
    if (status) status[k] = st != RICH_OK ? st : sst[k];
    if (info) info[k] = st == RICH_OK && steps[k] > 0 ? inf[k] : richards_step_info{};
  }
  return st;
}

richards_status richards_batcher_advance(richards_batcher* b, richards_ctx* const* ctxs, int n, const double* dt,
                                         const int* scheme, int* steps_left, int max_ticks, int* steps_done,
                                         richards_status* status, richards_step_info* info) {
  if (!b || !ctxs || !dt || !scheme || !steps_left || n < 1) return RICH_EINVAL;
  for (int k = 0; k < n; ++k)
    if (steps_left[k] < 0) return bfail(b, RICH_EINVAL, "negative steps_left");
  TRY_B(batch_check(b, ctxs, n, dt, scheme));
  std::vector<int> want(steps_left, steps_left + n), steps(n, 0);
  std::vector<richards_status> sst(n, RICH_OK);
  std::vector<richards_step_info> inf(n);
  const richards_status st = batch_call(b, ctxs, n, dt, scheme, want, false, max_ticks, steps, sst, inf);
  for (int k = 0; k < n; ++k) {
    if (st == RICH_OK) steps_left[k] = want[k];
    if (steps_done) steps_done[k] = st == RICH_OK ? steps[k] : 0;
    if (status) status[k] = st != RICH_OK ? st : sst[k];
    if (info) info[k] = st == RICH_OK && steps[k] > 0 ? inf[k] : richards_step_info{};
  }
  return st;
}

long long richards_device_bytes(const richards_grid* grid, const richards_opts* opts, int soil_fields, int sink) {
  if (!grid || !opts || grid->dim < 1 || grid->dim > 3) return -1;
  long long n[3] = {grid->n[0], grid->n[1], grid->n[2]};
  for (int a = 0; a < 3; ++a)
    if (n[a] < 1) return -1;
  const bool mixed = opts->precision >= 1;
  const long long N = n[0] * n[1] * n[2];
  long long bytes = 2 * N * 8 + (mixed ? 3 * N * 8 : 0) + (soil_fields > 0 ? N * 8 : 0);   // psi^n, psi^{n-1}, caches, Ks
  int levels = 0;
  for (;;) {
    const long long cells = n[0] * n[1] * n[2];
    long long faces = 0;
    for (int a = 0; a < grid->dim; ++a) faces += 2 * (cells / n[a]);
    bytes += cells * 8 * (5 + (soil_fields > 0 ? 2 : 0) + (sink ? 1 : 0)) + faces * 8;
    if (mixed) bytes += cells * 4 * (6 + (soil_fields > 0 ? 2 : 0) + (sink ? 1 : 0)) + faces * 4;
    for (int a = 0; a < 3; ++a) bytes += (n[a] * 5 + 13 * ((n[a] + 1) / 2)) * 8;   // transfer tables (bound)
    ++levels;
    const long long mx = std::max(n[0], std::max(n[1], n[2]));
    if (mx <= opts->coarsest_max_n || (opts->max_levels > 0 && levels >= opts->max_levels) || levels >= MAXLEV) break;
    for (int a = 0; a < 3; ++a) n[a] = n[a] > 1 ? (n[a] + 1) / 2 : 1;
  }
  return bytes;
}

richards_status richards_get_level(richards_ctx* c, int level, int which, double* out, long long n) {
  if (!c || !out || level < 0 || level >= c->nlev) return RICH_EINVAL;
  if (c->busy.load()) return fail(c, RICH_EBUSY, "context busy: a batch is running on it");
  HLevel& H = c->L[level];
  const double* src = nullptr;
  long long cnt = H.ncell;
  switch (which) {
    case 0: src = H.u; break;
    case 1: src = H.g; break;
    case 2: src = H.Kc; break;
    case 3: src = c->het_p1 ? H.p1 : nullptr; break;
    case 4: src = c->het_p2 ? H.p2 : nullptr; break;
    case 5: src = c->sink.enabled ? H.smax : nullptr; break;
    case 6: src = H.ubar; break;
    case 7: src = H.d; break;
    case 8: {                         // material index (layered soils)
      if (!c->layered) return fail(c, RICH_EINVAL, "array not available");
      if (n != H.ncell) return fail(c, RICH_EINVAL, "size mismatch");
      std::vector<uint8_t> m(H.ncell);
      CK(cudaMemcpyAsync(m.data(), H.mat, H.ncell, cudaMemcpyDeviceToHost, c->s));
      CK(cudaStreamSynchronize(c->s));
      for (long long i = 0; i < H.ncell; ++i) out[i] = m[i];
      return RICH_OK;
    }
    default:
      if (which >= 10 && which < 16) { src = H.kb[which - 10]; cnt = H.nface[which - 10]; }
  }
  if (!src) return fail(c, RICH_EINVAL, "array not available");
  if (n != cnt) return fail(c, RICH_EINVAL, "size mismatch");
  CK(cudaMemcpyAsync(out, src, sizeof(double) * cnt, cudaMemcpyDeviceToHost, c->s));
  CK(cudaStreamSynchronize(c->s));
  return RICH_OK;
}

richards_status richards_set_level(richards_ctx* c, int level, int which, const double* in, long long n) {
  if (!c || !in || level < 0 || level >= c->nlev || (which != 0 && which != 1)) return RICH_EINVAL;
  if (c->busy.load()) return fail(c, RICH_EBUSY, "context busy: a batch is running on it");
  HLevel& H = c->L[level];
  if (n != H.ncell) return fail(c, RICH_EINVAL, "size mismatch");
  CK(cudaMemcpyAsync(which == 0 ? H.u : H.g, in, sizeof(double) * n, cudaMemcpyHostToDevice, c->s));
  CK(cudaStreamSynchronize(c->s));
  return RICH_OK;
}

richards_status richards_sweep(richards_ctx* c, int level, int color) {
  if (!c || level < 0 || level >= c->nlev || color < -1 || color > 1) return RICH_EINVAL;
  if (c->busy.load()) return fail(c, RICH_EBUSY, "context busy: a batch is running on it");
  if (!c->prepared) return fail(c, RICH_EINVAL, "call richards_prepare first");
  const Level<double> L = view64(c, level);
  const Phys<double> P = phys<double>(c);
  if (c->opts.ordering == 0) {
    if (color != -1) return fail(c, RICH_EINVAL, "lexicographic ordering: only whole sweeps (color -1)");
    rich::sweep_lex64(L, P, c->soil.model, c->s);
  } else {
    if (color != 1) rich::sweep64(L, P, c->soil.model, 0, c->s);
    if (color != 0) rich::sweep64(L, P, c->soil.model, 1, c->s);
  }
  TRY(check_launch(c));
  CK(cudaStreamSynchronize(c->s));
  return RICH_OK;
}

richards_status richards_residual(richards_ctx* c, int level, double* norm) {
  if (!c || level < 0 || level >= c->nlev) return RICH_EINVAL;
  if (c->busy.load()) return fail(c, RICH_EBUSY, "context busy: a batch is running on it");
  if (!c->prepared) return fail(c, RICH_EINVAL, "call richards_prepare first");
  double nr;
  TRY(norm64(c, level, &nr));
  if (norm) *norm = nr;
  return RICH_OK;
}

richards_status richards_restrict_tau(richards_ctx* c, int level) {
  if (!c || level < 0 || level + 1 >= c->nlev) return RICH_EINVAL;
  if (c->busy.load()) return fail(c, RICH_EBUSY, "context busy: a batch is running on it");
  if (!c->prepared) return fail(c, RICH_EINVAL, "call richards_prepare first");
  const Level<double> F = view64(c, level), C = view64(c, level + 1);
  const Phys<double> P = phys<double>(c);
  rich::residual64(F, P, c->soil.model, nullptr, c->s);
  rich::restrict64(F, C, xfer64(c, level), F.u, F.d, C.ubar, C.d, c->s);
  rich::tau64(C, P, c->soil.model, c->s);
  TRY(check_launch(c));
  CK(cudaStreamSynchronize(c->s));
  return RICH_OK;
}

richards_status richards_prolong(richards_ctx* c, int level) {
  if (!c || level < 0 || level + 1 >= c->nlev) return RICH_EINVAL;
  if (c->busy.load()) return fail(c, RICH_EBUSY, "context busy: a batch is running on it");
  rich::prolong64(view64(c, level), view64(c, level + 1), xfer64(c, level), c->s);
  TRY(check_launch(c));
  CK(cudaStreamSynchronize(c->s));
  return RICH_OK;
}

richards_status richards_vcycle(richards_ctx* c) {
  if (!c) return RICH_EINVAL;
  if (c->busy.load()) return fail(c, RICH_EBUSY, "context busy: a batch is running on it");
  if (!c->prepared) return fail(c, RICH_EINVAL, "call richards_prepare first");
  vcycle64(c, 0);
  TRY(check_launch(c));
  CK(cudaStreamSynchronize(c->s));
  return RICH_OK;
}

richards_status richards_profile(richards_ctx* c, int enable) {
  if (!c) return RICH_EINVAL;
  if (c->busy.load()) return fail(c, RICH_EBUSY, "context busy: a batch is running on it");
  if (enable) {
    prof_flush(c);
    c->prof_agg.clear();
  }
  c->harvest = nullptr;
  c->prof = enable;
  return RICH_OK;
}

int richards_profile_read(richards_ctx* c, richards_kernel_stat* out, int max) {
  if (!c || (!out && max > 0)) return -1;
  prof_flush(c);
  cudaStreamSynchronize(c->s);
  graph_harvest(c);
  int k = 0;
  for (const auto& kv : c->prof_agg) {
    if (k >= max) break;
    richards_kernel_stat& r = out[k++];
    std::memset(&r, 0, sizeof(r));
    std::strncpy(r.name, kv.first.first.c_str(), sizeof(r.name) - 1);
    r.level = kv.first.second;
    r.launches = kv.second.launches;
    r.ms = kv.second.ms;
    r.cells = kv.second.cells;
  }
  return k;
}

}  // extern "C"
