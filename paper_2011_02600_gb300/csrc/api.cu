// C ABI (include/sbp.h): grid handle, validation, stage sequencing.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "launch.h"
#include "sbp.h"
#include "source_weights.h"

#include <nvtx3/nvToolsExt.h>

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(SBP_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Carpenter & Kennedy (1994) five-stage 2N-storage fourth-order coefficients.
const double kRkA[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                        -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
const double kRkB[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                        1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                        2277821191437.0 / 14882151754819.0};

// Stage times c_k: total weight of dt f_j in the state seen by stage k
// (row sums of the equivalent Butcher tableau), so that they are consistent
// with A and B to rounding.
void rk_stage_times(double c[5]) {
  double reg[5] = {0, 0, 0, 0, 0}, acc[5] = {0, 0, 0, 0, 0};
  for (int k = 0; k < 5; ++k) {
    double s = 0;
    for (int j = 0; j < 5; ++j) s += acc[j];
    c[k] = s;
    for (int j = 0; j < 5; ++j) reg[j] = kRkA[k] * reg[j] + (j == k ? 1.0 : 0.0);
    for (int j = 0; j < 5; ++j) acc[j] += kRkB[k] * reg[j];
  }
}

// Properties of an operator code: the upwind orders 2 to 7 of Table 1 and the traditional
// operators kTraditional + 2, 4, 6 of Table 2.  b: closure rows at each end; reach:
// max(r, q) of the interior stencil; w0: first norm weight; metric_order: the upwind order
// whose D_c = (D+ + D-)/2 forms the metric terms; accuracy: the design order (the source's
// moment conditions use it).
struct OpInfo {
  bool ok = false;
  int b = 0, reach = 0, metric_order = 0, accuracy = 0;
  double w0 = 0.0;
  bool adjoint = false;  // the adjoint kernels are built for this operator
};
template <int O>
OpInfo op_info_of(int accuracy, int metric_order, bool adjoint) {
  OpInfo I;
  I.ok = true;
  I.b = sbp::OpCoef<O>::b;
  I.reach = sbp::OpCoef<O>::r > sbp::OpCoef<O>::q ? sbp::OpCoef<O>::r : sbp::OpCoef<O>::q;
  I.w0 = sbp::OpCoef<O>::w(0);
  I.metric_order = metric_order;
  I.accuracy = accuracy;
  I.adjoint = adjoint;
  return I;
}
OpInfo op_info(int order) {
  switch (order) {
    case 2: return op_info_of<2>(2, 2, true);
    case 3: return op_info_of<3>(3, 3, false);
    case 4: return op_info_of<4>(4, 4, true);
    case 5: return op_info_of<5>(5, 5, false);
    case 6: return op_info_of<6>(6, 6, true);
    case 7: return op_info_of<7>(7, 7, false);
    case sbp::kTraditional + 2: return op_info_of<sbp::kTraditional + 2>(2, 2, false);
    case sbp::kTraditional + 4: return op_info_of<sbp::kTraditional + 4>(4, 4, false);
    case sbp::kTraditional + 6: return op_info_of<sbp::kTraditional + 6>(6, 6, false);
    default: return OpInfo{};
  }
}
int closure_b(int order) { return op_info(order).b; }

// Norm weight w(pos) of the operator `order` on N nodes (H = h diag(w)).
double norm_weight_any(int order, int pos, int N) {
  switch (order) {
    case 2: return sbp::norm_weight<2>(pos, N);
    case 3: return sbp::norm_weight<3>(pos, N);
    case 4: return sbp::norm_weight<4>(pos, N);
    case 5: return sbp::norm_weight<5>(pos, N);
    case 6: return sbp::norm_weight<6>(pos, N);
    case 7: return sbp::norm_weight<7>(pos, N);
    case sbp::kTraditional + 2: return sbp::norm_weight<sbp::kTraditional + 2>(pos, N);
    case sbp::kTraditional + 4: return sbp::norm_weight<sbp::kTraditional + 4>(pos, N);
    case sbp::kTraditional + 6: return sbp::norm_weight<sbp::kTraditional + 6>(pos, N);
    default: return 0.0;
  }
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  return fn;
}

}  // namespace

namespace sbp {
void set_last_error(const char* msg) { g_last_error = msg; }
}  // namespace sbp

struct SbpGrid {
  SbpGridDesc desc;
  sbp::Dims dims;
  int elem;
  void* q[2] = {nullptr, nullptr};
  void* dq = nullptr;
  void* met = nullptr;
  void* mat = nullptr;
  int cur = 0;
  bool bound = false, material = false;
  double t = 0.0;
  long long step = 0;
  double rkc[5];
  // internal device buffers
  double* partial = nullptr;
  double* eout = nullptr;
  unsigned* status = nullptr;
  int nb = 1;  // independent states bound together (sbp_set_batch)
  long long* src_off = nullptr;
  double* src_w = nullptr;
  int src_n = 0;
  SbpSource src;
  int32_t* rec_off = nullptr;
  int rec_n = 0;
  void* traces = nullptr;
  bool traces_owned = false;  // traces allocated by the library (sbp_set_receivers with traces = NULL)
  int n_t = 0;
  bool use_tiled = true;
  sbp::SlabS slab;         // s-slab of a decomposed block (sbp_set_slab); default: the whole block
  const void* iface[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};  // other blocks' traces
  void* sclose = nullptr;  // tiled kernel scratch (s-closure sums), owned by the library
  // topography map (found by sbp_set_material): the tiled forward stage reads a_q,x and a_s only
  unsigned long long* topo_dev = nullptr;  // detection scratch (one word)
  bool topo = false;
  double ar_ratio = 0.0;  // a_r,y / a_q,x
  int map_path = SBP_MAP_AUTO;
  // tensor maps of the tiled stage kernel, per state buffer (q0, q1)
  bool tma_ok[2] = {false, false};
  sbp::TmaSet tma[2];
  // tensor maps of other inputs of the tiled kernel (the adjoint's yhat and stage states), by pointer
  std::vector<std::pair<const void*, sbp::TmaSet>> tma_cache;
  // optional per-kernel CUDA-event timing (kind 0 = tiled stage, 1 = general stage, 2 = adjoint stage)
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_pending;
};

namespace {

// NVTX range around a C-ABI call (shows in nsys/ncu timelines; free when no tool listens).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

// Nodes of face f (0..5) of the grid.
long long face_nodes(const SbpGrid* g, int f) {
  const int xi = f / 2;
  return xi == 0 ? (long long)g->desc.nr * g->desc.ns
                 : xi == 1 ? (long long)g->desc.nq * g->desc.ns : (long long)g->desc.nq * g->desc.nr;
}

bool has_interface(const SbpGrid* g) {
  for (int f = 0; f < 6; ++f)
    if (g->desc.bc_kind[f] == SBP_BC_INTERFACE) return true;
  return false;
}

// Every interface face needs the other block's trace before a stage can run.
int check_interfaces(const SbpGrid* g) {
  for (int f = 0; f < 6; ++f)
    if (g->desc.bc_kind[f] == SBP_BC_INTERFACE && !g->iface[f])
      return fail(SBP_ERR_STATE, "face %d is an interface without the other block's trace (sbp_set_interface)", f);
  return SBP_OK;
}

// Elements of the tiled kernel's s-closure scratch per state: 2 ends x b rows x 6 planes.
long long sclose_elems(const SbpGrid* g) { return 2LL * closure_b(g->desc.order) * 6 * g->dims.plane; }

// The whole grid as one box (the general kernel's work list).
sbp::BoxList whole_grid(const SbpGrid* g) {
  sbp::BoxList L;
  L.n = 1;
  L.b[0] = sbp::Box{0, g->desc.nq, 0, g->desc.nr, 0, g->desc.ns};
  L.off[0] = 0;
  L.off[1] = (long long)g->desc.nq * g->desc.nr * g->desc.ns;
  return L;
}

// The tiled forward stage reads the topography map's 4 metric fields where the metrics are
// those of such a map (sbp_set_material), the path is automatic (sbp_set_map_path) and the
// variant is built for the operator (upwind orders 2, 4, 6).
bool uses_topography(const SbpGrid* g) {
  const int o = g->desc.order;
  return g->topo && g->map_path == SBP_MAP_AUTO && (o == 2 || o == 4 || o == 6);
}

template <typename T>
sbp::StageArgs<T> make_args(const SbpGrid* g, const void* q, void* qout, int mode, double a, double bcoef,
                            double dt, int nb = 1) {
  sbp::StageArgs<T> A{};
  A.nb = nb;
  A.bstride = 9 * g->dims.fs;
  A.q = (const T*)q;
  A.qout = (T*)qout;
  A.dq = (T*)g->dq;
  A.met = (const T*)g->met;
  A.mat = (const T*)g->mat;
  A.d = g->dims;
  A.rk_a = (T)a;
  A.rk_b = (T)bcoef;
  A.dt = (T)dt;
  A.mode = mode;
  A.status = g->status;
  A.sclose = (T*)g->sclose;
  A.sc_bstride = sclose_elems(g);
  A.slab = g->slab;
  A.map = uses_topography(g) ? 1 : 0;
  A.ar_ratio = (T)g->ar_ratio;
  // spacing along s: that of the whole block when the grid is one of its slabs
  const int N[3] = {g->desc.nq, g->desc.nr, g->slab.ns_global > 0 ? g->slab.ns_global : g->desc.ns};
  for (int f = 0; f < 6; ++f) {
    A.bc_kind[f] = g->desc.bc_kind[f];
    A.bc_gamma[f] = (T)g->desc.bc_gamma[f];
    A.ifc.other[f] = (const T*)g->iface[f];
    A.ifc.n_face[f] = face_nodes(g, f);
  }
  const double w0 = op_info(g->desc.order).w0;
  for (int x = 0; x < 3; ++x) {
    A.inv_h[x] = (T)(N[x] - 1);
    A.inv_h0[x] = (T)((double)(N[x] - 1) / w0);
    A.h[x] = (T)(1.0 / (N[x] - 1));
  }
  return A;
}

cudaEvent_t pool_event(SbpGrid* g) {
  if (!g->ev_pool.empty()) {
    cudaEvent_t e = g->ev_pool.back();
    g->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Record events around one kernel launch when timing is on.
struct TimedLaunch {
  SbpGrid* g;
  int kind;
  cudaStream_t st;
  cudaEvent_t a = nullptr, b = nullptr;
  TimedLaunch(SbpGrid* g_, int kind_, cudaStream_t st_) : g(g_), kind(kind_), st(st_) {
    if (g->timing) {
      a = pool_event(g);
      b = pool_event(g);
      cudaEventRecord(a, st);
    }
  }
  void done() {
    if (g->timing && a && b) {
      cudaEventRecord(b, st);
      g->ev_pending.push_back({kind, {a, b}});
    }
  }
};

// Tensor maps for the tiled kernel's tile loads (kernels_tiled.cu): the state
// (box 40 x 16 x 1 x 9), the metric vectors a_q (40 x 8 x 1 x 3), a_r (32 x 16 x 1 x 3),
// a_s (32 x 8 x 1 x 3) and the coefficients (32 x 8 x 1 x 3).  Out-of-range elements
// are filled with zeros.
int encode_maps(const SbpGrid* g, const void* q, int nb, sbp::TmaSet* out) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return fail(SBP_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  const sbp::Dims& d = g->dims;
  const CUtensorMapDataType dt = g->elem == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
  auto one = [&](CUtensorMap* m, const void* base, int nf, unsigned bx, unsigned by, unsigned bf) -> int {
    const cuuint64_t dims[4] = {(cuuint64_t)d.nq, (cuuint64_t)d.nr, (cuuint64_t)d.ns, (cuuint64_t)nf};
    const cuuint64_t strides[3] = {(cuuint64_t)d.ldq * g->elem, (cuuint64_t)d.plane * g->elem,
                                   (cuuint64_t)d.fs * g->elem};
    const cuuint32_t box[4] = {bx, by, 1, bf};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = enc(m, dt, 4, const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? SBP_OK : fail(SBP_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  };
  int rc = one(&out->state, q, 9 * nb, 40, 16, 9);
  if (!rc) rc = one(&out->met_q, g->met, 9, 40, 8, 3);
  if (!rc) rc = one(&out->met_r, g->met, 9, 32, 16, 3);
  if (!rc) rc = one(&out->met_s, g->met, 9, 32, 8, 3);
  if (!rc) rc = one(&out->mat, g->mat, 3, 32, 8, 3);
  if (!rc) rc = one(&out->met_j, g->met, 9, 40, 16, 1);
  if (!rc) rc = one(&out->dq, g->dq, 9 * g->nb, 32, 8, 9);
  return rc;
}

// Tensor maps of an input buffer of the tiled kernel holding the grid's B states, encoded
// once per pointer.
int cached_maps(SbpGrid* g, const void* p, const sbp::TmaSet** out) {
  for (auto& c : g->tma_cache)
    if (c.first == p) {
      *out = &c.second;
      return SBP_OK;
    }
  if (g->tma_cache.size() >= 16) g->tma_cache.clear();
  g->tma_cache.emplace_back(p, sbp::TmaSet{});
  if (int rc = encode_maps(g, p, g->nb, &g->tma_cache.back().second)) {
    g->tma_cache.pop_back();
    return rc;
  }
  *out = &g->tma_cache.back().second;
  return SBP_OK;
}

template <typename T>
int run_stage_kernels(SbpGrid* g, const void* q, void* qout, int mode, double a, double bcoef, double dt,
                      cudaStream_t st, int nb = 1) {
  if (g->slab.ns_global > 0 && !g->use_tiled)
    return fail(SBP_ERR_UNSUPPORTED, "a slab grid runs the tiled kernel only (sbp_set_kernel_path(0))");
  if (int rc = check_interfaces(g)) return rc;
  sbp::StageArgs<T> A = make_args<T>(g, q, qout, mode, a, bcoef, dt, nb);
  if (g->use_tiled) {
    sbp::TmaSet local;
    const sbp::TmaSet* tm = &local;
    const int which = nb == g->nb ? (q == g->q[0] ? 0 : q == g->q[1] ? 1 : -1) : -1;
    if (which >= 0) {
      if (!g->tma_ok[which]) {
        if (int rc = encode_maps(g, q, nb, &g->tma[which])) return rc;
        g->tma_ok[which] = true;
      }
      tm = &g->tma[which];
    } else if (int rc = encode_maps(g, q, nb, &local)) {
      return rc;
    }
    TimedLaunch ti(g, 0, st);
    cudaError_t e = sbp::launch_stage_tiled<T>(A, g->desc.order, *tm, st);
    if (e != cudaSuccess) return cuda_fail(e, "stage (tiled)");
    ti.done();
    return SBP_OK;
  }
  TimedLaunch ts(g, 1, st);
  cudaError_t e = sbp::launch_stage_general<T>(A, g->desc.order, whole_grid(g), st);
  if (e != cudaSuccess) return cuda_fail(e, "stage (general)");
  ts.done();
  return SBP_OK;
}

double stf_value(const SbpSource& s, double t) {
  if (s.stf == 0) {
    const double a = M_PI * s.f0 * (t - s.t0);
    return (1.0 - 2.0 * a * a) * exp(-a * a);
  }
  return t > 0 ? t / (s.T * s.T) * exp(-t / s.T) : 0.0;
}

template <typename T>
int stage_impl(SbpGrid* g, int k, double dt, cudaStream_t st) {
  const void* qin = g->q[g->cur];
  void* qout = g->q[1 - g->cur];
  const int mode = k == 0 ? sbp::kModeStage0 : sbp::kModeStage;
  int rc = run_stage_kernels<T>(g, qin, qout, mode, kRkA[k], kRkB[k], dt, st, g->nb);
  if (rc) return rc;
  if (g->src_n > 0) {
    const double gdt = stf_value(g->src, g->t + g->rkc[k] * dt) * dt;
    cudaError_t e = sbp::launch_source<T>((T*)qout, (T*)g->dq, g->dims, g->src_off, g->src_w, g->src_n, gdt,
                                          kRkB[k], mode, st);
    if (e != cudaSuccess) return cuda_fail(e, "source");
  }
  g->cur = 1 - g->cur;
  return SBP_OK;
}

int check_ready(const SbpGrid* g) {
  if (!g) return fail(SBP_ERR_ARG, "null grid");
  if (!g->bound) return fail(SBP_ERR_STATE, "buffers not bound (sbp_bind)");
  return SBP_OK;
}

}  // namespace

namespace {
template <typename T>
int adjoint_impl(SbpGrid* g, int mode, int stage, double dt, const void* u, void* ubar, const void* win, void* wbar,
                 void* scratch, const double* rlmj, double* grad, cudaStream_t st) {
  sbp::AdjArgs<T> A{};
  A.nb = g->nb;
  A.bstride = 9 * g->dims.fs;
  A.ubar_next = mode == 1 ? (const T*)ubar : nullptr;
  A.ubar_out = (T*)ubar;
  A.wbar_in = (const T*)win;
  A.wbar = (T*)wbar;
  A.yhat = (T*)scratch;
  A.u = (const T*)u;
  A.met = (const T*)g->met;
  A.mat = (const T*)g->mat;
  A.rlmj = rlmj;
  A.grad = grad;
  A.d = g->dims;
  A.rk_a = mode == 1 ? (T)kRkA[stage] : T(0);
  A.rk_b = mode == 1 ? (T)kRkB[stage] : T(0);
  A.dt = (T)dt;
  A.mode = mode;
  sbp::StageArgs<T> S = make_args<T>(g, nullptr, nullptr, 0, 0, 0, 0);
  for (int f = 0; f < 6; ++f) {
    A.bc_kind[f] = S.bc_kind[f];
    A.bc_gamma[f] = S.bc_gamma[f];
  }
  for (int x = 0; x < 3; ++x) {
    A.inv_h[x] = S.inv_h[x];
    A.inv_h0[x] = S.inv_h0[x];
  }
  TimedLaunch ta(g, 2, st);
  if (!g->use_tiled) {
    cudaError_t e = sbp::launch_adjoint<T>(A, g->desc.order, st);
    if (e != cudaSuccess) return cuda_fail(e, "adjoint");
  } else {
    // prep (Wb_k, yhat), then the tiled gradient pass on U_k and the tiled L^T pass on yhat
    cudaError_t e = sbp::launch_adjoint_prep<T>(A, g->desc.order, st);
    if (e != cudaSuccess) return cuda_fail(e, "adjoint prep");
    sbp::StageArgs<T> S2 = make_args<T>(g, nullptr, nullptr, mode == 1 ? sbp::kModeStage : sbp::kModeRhs,
                                        mode == 1 ? kRkA[stage] : 0.0, 0.0, dt, g->nb);
    S2.ubar_next = A.ubar_next;
    S2.ubar_out = A.ubar_out;
    S2.wbar = A.wbar;
    S2.yhat = A.yhat;
    S2.rlmj = rlmj;
    S2.grad = grad;
    if (grad && u) {
      const sbp::TmaSet* tu = nullptr;
      if (int rc = cached_maps(g, u, &tu)) return rc;
      S2.q = (const T*)u;
      e = sbp::launch_adjoint_tiled<T>(S2, g->desc.order, 2, *tu, st);
      if (e != cudaSuccess) return cuda_fail(e, "adjoint gradient (tiled)");
    }
    const sbp::TmaSet* ty = nullptr;
    if (int rc = cached_maps(g, scratch, &ty)) return rc;
    S2.q = (const T*)scratch;
    e = sbp::launch_adjoint_tiled<T>(S2, g->desc.order, 1, *ty, st);
    if (e != cudaSuccess) return cuda_fail(e, "adjoint (tiled)");
  }
  ta.done();
  return SBP_OK;
}

// One whole adjoint step (stages 4..0) on the tiled kernel, the prep of each stage k < 4 fused
// into the L^T pass of stage k + 1 (pointwise there); scratch holds two yhat buffers used in turn.
template <typename T>
int adjoint_step_impl(SbpGrid* g, double dt, const void* u5, void* ubar, void* wbar, void* scratch,
                      const double* rlmj, double* grad, cudaStream_t st) {
  const long long grp = 9LL * g->nb * g->dims.fs;  // elements of one group of B states
  T* y[2] = {(T*)scratch, (T*)scratch + grp};
  for (int k = 4; k >= 0; --k) {
    TimedLaunch ta(g, 2, st);
    T* yc = y[(4 - k) & 1];
    if (k == 4) {
      // the prep of stage 4 on its own: Ub_5 holds the step's receiver sources
      sbp::AdjArgs<T> A{};
      A.nb = g->nb;
      A.bstride = 9 * g->dims.fs;
      A.ubar_next = (const T*)ubar;
      A.ubar_out = (T*)ubar;
      A.wbar_in = (const T*)wbar;
      A.wbar = (T*)wbar;
      A.yhat = yc;
      A.mat = (const T*)g->mat;
      A.d = g->dims;
      A.rk_b = (T)kRkB[4];
      A.mode = 1;
      sbp::StageArgs<T> S = make_args<T>(g, nullptr, nullptr, 0, 0, 0, 0);
      for (int x = 0; x < 3; ++x) A.inv_h[x] = S.inv_h[x];
      cudaError_t e = sbp::launch_adjoint_prep<T>(A, g->desc.order, st);
      if (e != cudaSuccess) return cuda_fail(e, "adjoint prep");
    }
    sbp::StageArgs<T> S2 = make_args<T>(g, nullptr, nullptr, sbp::kModeStage, kRkA[k], 0.0, dt, g->nb);
    S2.ubar_next = (const T*)ubar;
    S2.ubar_out = (T*)ubar;
    S2.wbar = (T*)wbar;
    S2.yhat = yc;
    S2.rlmj = rlmj;
    S2.grad = grad;
    if (grad) {
      const T* uk = (const T*)u5 + k * grp;
      const sbp::TmaSet* tu = nullptr;
      if (int rc = cached_maps(g, uk, &tu)) return rc;
      S2.q = uk;
      cudaError_t e = sbp::launch_adjoint_tiled<T>(S2, g->desc.order, 2, *tu, st);
      if (e != cudaSuccess) return cuda_fail(e, "adjoint gradient (tiled)");
    }
    const sbp::TmaSet* ty = nullptr;
    if (int rc = cached_maps(g, yc, &ty)) return rc;
    S2.q = yc;
    S2.yhat_next = k > 0 ? y[(5 - k) & 1] : nullptr;
    S2.rk_b_next = k > 0 ? (T)kRkB[k - 1] : T(0);
    cudaError_t e = sbp::launch_adjoint_tiled<T>(S2, g->desc.order, 1, *ty, st);
    if (e != cudaSuccess) return cuda_fail(e, "adjoint (tiled)");
    ta.done();
  }
  return SBP_OK;
}

// Copy the 9 B state fields between the bound buffer dev (grid layout) and a caller buffer
// ext: host or device memory (SBP_MEM_HOST), in the grid layout (9 B fields of fs elements) or
// packed [field][s][r][q] (SBP_LAYOUT_DENSE).  A copy to host memory synchronises the stream.
int copy_state(SbpGrid* g, void* dev, const void* ext, int flags, bool in, cudaStream_t st) {
  const bool host = (flags & SBP_MEM_HOST) != 0;
  const bool dense = (flags & SBP_LAYOUT_DENSE) != 0;
  const cudaMemcpyKind kind = host ? (in ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost) : cudaMemcpyDeviceToDevice;
  const int nf = 9 * g->nb;
  const size_t e = (size_t)g->elem;
  cudaError_t err = cudaSuccess;
  if (!dense) {
    const size_t bytes = (size_t)nf * g->dims.fs * e;
    err = in ? cudaMemcpyAsync(dev, ext, bytes, kind, st) : cudaMemcpyAsync(const_cast<void*>(ext), dev, bytes, kind, st);
  } else {
    // one pitched copy per field: nr*ns rows of nq elements, row pitch ldq in the grid layout
    const size_t row = (size_t)g->desc.nq * e, pitch = (size_t)g->dims.ldq * e;
    const size_t rows = (size_t)g->desc.nr * g->desc.ns, field = row * rows;
    for (int f = 0; f < nf && err == cudaSuccess; ++f) {
      char* d = (char*)dev + (size_t)f * g->dims.fs * e;
      char* x = (char*)const_cast<void*>(ext) + (size_t)f * field;
      err = in ? cudaMemcpy2DAsync(d, pitch, x, row, row, rows, kind, st)
               : cudaMemcpy2DAsync(x, row, d, pitch, row, rows, kind, st);
    }
  }
  if (err == cudaSuccess && host && !in && !(flags & SBP_MEM_ASYNC)) err = cudaStreamSynchronize(st);
  return err == cudaSuccess ? SBP_OK : cuda_fail(err, in ? "state upload" : "state download");
}

}  // namespace

extern "C" {

const char* sbp_last_error(void) { return g_last_error.c_str(); }

int sbp_min_nodes(int32_t order, int32_t* out) {
  const OpInfo I = op_info(order);
  if (!I.ok)
    return fail(SBP_ERR_ARG, "order must be 2..7 (upwind, Table 1) or %d, %d, %d (traditional, Table 2)",
                SBP_TRADITIONAL + 2, SBP_TRADITIONAL + 4, SBP_TRADITIONAL + 6);
  if (!out) return fail(SBP_ERR_ARG, "null output");
  // the metric terms apply the upwind pair of the operator's order: its size bound holds too
  const OpInfo Im = op_info(I.metric_order);
  const int own = 2 * I.b + I.reach, met = 2 * Im.b + Im.reach;
  *out = own > met ? own : met;
  return SBP_OK;
}

int sbp_rk_coefficients(double* A, double* B, double* C) {
  double c[5];
  rk_stage_times(c);
  for (int k = 0; k < 5; ++k) {
    if (A) A[k] = kRkA[k];
    if (B) B[k] = kRkB[k];
    if (C) C[k] = c[k];
  }
  return SBP_OK;
}

int sbp_create_grid(const SbpGridDesc* desc, SbpGrid** out) {
  if (!desc || !out) return fail(SBP_ERR_ARG, "null argument");
  *out = nullptr;
  int32_t nmin;
  if (sbp_min_nodes(desc->order, &nmin)) return SBP_ERR_ARG;
  if (desc->nq < nmin || desc->nr < nmin || desc->ns < nmin)
    return fail(SBP_ERR_ARG, "order %d needs at least %d nodes per axis (got %d x %d x %d)", desc->order, nmin,
                desc->nq, desc->nr, desc->ns);
  if (desc->precision != 32 && desc->precision != 64) return fail(SBP_ERR_ARG, "precision must be 32 or 64");
  for (int f = 0; f < 6; ++f) {
    if (desc->bc_kind[f] != SBP_BC_FREE && desc->bc_kind[f] != SBP_BC_CHAR && desc->bc_kind[f] != SBP_BC_INTERFACE)
      return fail(SBP_ERR_ARG, "face %d: unknown boundary kind %d", f, desc->bc_kind[f]);
    if (desc->bc_kind[f] == SBP_BC_CHAR && !(fabs(desc->bc_gamma[f]) <= 1.0))
      return fail(SBP_ERR_ARG, "face %d: gamma must lie in [-1, 1]", f);
  }
  const int elem = desc->precision == 32 ? 4 : 8;
  const int align = 128 / elem;
  const long long ldq = ((long long)desc->nq + align - 1) / align * align;
  const long long plane = ldq * desc->nr;
  long long fs = plane * desc->ns;
  fs = (fs + 255) / 256 * 256;  // 256-byte aligned field starts for either precision
  if (fs >= (1LL << 31) || plane >= (1LL << 31))
    return fail(SBP_ERR_ARG, "grid too large: %lld elements per field (limit 2^31)", fs);
  SbpGrid* g = new SbpGrid();
  g->desc = *desc;
  g->elem = elem;
  g->dims = sbp::Dims{desc->nq, desc->nr, desc->ns, (int)ldq, (int)plane, fs};
  rk_stage_times(g->rkc);
  g->use_tiled = true;
  *out = g;
  return SBP_OK;
}

int sbp_destroy(SbpGrid* g) {
  if (!g) return SBP_OK;
  for (auto& p : g->ev_pending) {
    cudaEventDestroy(p.second.first);
    cudaEventDestroy(p.second.second);
  }
  for (auto e : g->ev_pool) cudaEventDestroy(e);
  cudaFree(g->partial);
  cudaFree(g->eout);
  cudaFree(g->status);
  cudaFree(g->src_off);
  cudaFree(g->src_w);
  cudaFree(g->rec_off);
  if (g->traces_owned) cudaFree(g->traces);
  cudaFree(g->sclose);
  cudaFree(g->topo_dev);
  delete g;
  return SBP_OK;
}

int sbp_layout(const SbpGrid* g, int64_t* ldq, int64_t* fs, int64_t* elem) {
  if (!g) return fail(SBP_ERR_ARG, "null grid");
  if (ldq) *ldq = g->dims.ldq;
  if (fs) *fs = g->dims.fs;
  if (elem) *elem = g->elem;
  return SBP_OK;
}

int sbp_bind(SbpGrid* g, void* q0, void* q1, void* dq, void* met, void* mat) {
  if (!g) return fail(SBP_ERR_ARG, "null grid");
  void* p[5] = {q0, q1, dq, met, mat};
  for (int i = 0; i < 5; ++i) {
    if (!p[i]) return fail(SBP_ERR_ARG, "buffer %d is null", i);
    if ((uintptr_t)p[i] % 256) return fail(SBP_ERR_ARG, "buffer %d is not 256-byte aligned", i);
    for (int j = 0; j < i; ++j)
      if (p[i] == p[j]) return fail(SBP_ERR_ARG, "buffers %d and %d alias", j, i);
  }
  g->q[0] = q0;
  g->q[1] = q1;
  g->dq = dq;
  g->met = met;
  g->mat = mat;
  g->cur = 0;
  g->tma_ok[0] = g->tma_ok[1] = false;
  g->tma_cache.clear();
  if (!g->partial) {
    cudaError_t e = cudaMalloc(&g->partial, sizeof(double) * sbp::energy_blocks());
    if (e == cudaSuccess) e = cudaMalloc(&g->eout, sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&g->status, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(g->status, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&g->topo_dev, sizeof(unsigned long long));
    if (e != cudaSuccess) return cuda_fail(e, "internal buffers");
  }
  if (!g->sclose) {
    cudaError_t e = cudaMalloc(&g->sclose, (size_t)sclose_elems(g) * g->nb * g->elem);
    if (e != cudaSuccess) return cuda_fail(e, "tiled kernel scratch");
  }
  g->bound = true;
  return SBP_OK;
}

int sbp_metrics(SbpGrid* g, const double* xyz, double* jmet, void* stream) {
  if (int rc = check_ready(g)) return rc;
  if (!xyz || !jmet) return fail(SBP_ERR_ARG, "null coordinate or metric buffer");
  // D_c of the metric operator reaches further than the central operators it serves: a slab's
  // inner ends must hold that many planes of coordinates
  const int mreach = op_info(op_info(g->desc.order).metric_order).reach;
  if ((g->slab.ghost_lo > 0 && g->slab.ghost_lo < mreach) || (g->slab.ghost_hi > 0 && g->slab.ghost_hi < mreach))
    return fail(SBP_ERR_ARG, "metrics on a slab need at least %d ghost planes at an inner end", mreach);
  cudaError_t e = sbp::launch_metrics(xyz, jmet, g->dims, op_info(g->desc.order).metric_order, g->status,
                                      (cudaStream_t)stream, g->slab);
  return e == cudaSuccess ? SBP_OK : cuda_fail(e, "metrics");
}

int sbp_set_material(SbpGrid* g, const double* jmet, const double* rlm, void* stream) {
  if (int rc = check_ready(g)) return rc;
  if (!jmet || !rlm) return fail(SBP_ERR_ARG, "null metric or material buffer");
  cudaError_t e = g->elem == 4 ? sbp::launch_material<float>(jmet, rlm, (float*)g->met, (float*)g->mat, g->dims,
                                                             g->status, (cudaStream_t)stream)
                               : sbp::launch_material<double>(jmet, rlm, (double*)g->met, (double*)g->mat, g->dims,
                                                              g->status, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "material");
  // topography map?  c = a_r,y / a_q,x at node 0, then every node within 1e-11 (relative) of
  // a_q = (a_q,x, 0, 0), a_r = (0, c a_q,x, 0).  The components that vanish for such a map come
  // out of D_c applied to the linear x and y as rounding noise that grows with the node count
  // (about 1e-13 of a_q,x on 1025 nodes); genuinely curvilinear maps are far above the bound.
  cudaStream_t st = (cudaStream_t)stream;
  const sbp::Dims& d = g->dims;
  double a0[2] = {0.0, 0.0};
  unsigned long long worst = ~0ull;
  e = cudaMemcpyAsync(&a0[0], jmet + 1 * d.fs, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&a0[1], jmet + 5 * d.fs, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  const double c = a0[1] / a0[0];
  g->topo = false;
  if (e == cudaSuccess && isfinite(c) && c > 0.0) {
    e = cudaMemsetAsync(g->topo_dev, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = sbp::launch_topography_check(jmet, d, c, g->topo_dev, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&worst, g->topo_dev, sizeof(worst), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    double w;
    memcpy(&w, &worst, sizeof(w));
    g->topo = e == cudaSuccess && w <= 1.0e-11;
    g->ar_ratio = c;
  }
  if (e != cudaSuccess) return cuda_fail(e, "topography check");
  g->material = true;
  return SBP_OK;
}

int sbp_set_map_path(SbpGrid* g, int32_t path) {
  if (!g) return fail(SBP_ERR_ARG, "null grid");
  if (path != SBP_MAP_AUTO && path != SBP_MAP_GENERAL) return fail(SBP_ERR_ARG, "map path must be 0 (auto) or 1 (general)");
  g->map_path = path;
  return SBP_OK;
}

int sbp_map_path(SbpGrid* g, int32_t* path) {
  if (!g || !path) return fail(SBP_ERR_ARG, "null argument");
  *path = uses_topography(g) && g->use_tiled ? SBP_MAP_TOPOGRAPHY : SBP_MAP_GENERAL;
  return SBP_OK;
}

int sbp_rhs(SbpGrid* g, const void* q, void* out, void* stream) {
  if (int rc = check_ready(g)) return rc;
  if (!g->material) return fail(SBP_ERR_STATE, "material not set (sbp_set_material)");
  if (!q || !out || q == out) return fail(SBP_ERR_ARG, "rhs needs distinct input and output buffers");
  return g->elem == 4 ? run_stage_kernels<float>(g, q, out, sbp::kModeRhs, 0, 0, 0, (cudaStream_t)stream)
                      : run_stage_kernels<double>(g, q, out, sbp::kModeRhs, 0, 0, 0, (cudaStream_t)stream);
}

int sbp_rk_stage(SbpGrid* g, int32_t stage, double dt, void* stream) {
  NvtxRange nvtx_range("sbp_rk_stage");
  if (int rc = check_ready(g)) return rc;
  if (!g->material) return fail(SBP_ERR_STATE, "material not set (sbp_set_material)");
  if (stage < 0 || stage > 4) return fail(SBP_ERR_ARG, "stage must be 0..4");
  if (!(dt > 0) || !isfinite(dt)) return fail(SBP_ERR_ARG, "dt must be positive and finite");
  return g->elem == 4 ? stage_impl<float>(g, stage, dt, (cudaStream_t)stream)
                      : stage_impl<double>(g, stage, dt, (cudaStream_t)stream);
}

int sbp_step_n(SbpGrid* g, int32_t n, double dt, void* stream) {
  NvtxRange nvtx_range("sbp_step_n");
  if (int rc = check_ready(g)) return rc;
  if (!g->material) return fail(SBP_ERR_STATE, "material not set (sbp_set_material)");
  if (n < 0) return fail(SBP_ERR_ARG, "negative step count");
  if (!(dt > 0) || !isfinite(dt)) return fail(SBP_ERR_ARG, "dt must be positive and finite");
  if (has_interface(g))
    return fail(SBP_ERR_UNSUPPORTED, "a grid with interface faces steps stage by stage (sbp_rk_stage), its "
                                     "traces refreshed before every stage");
  cudaStream_t st = (cudaStream_t)stream;
  for (int s = 0; s < n; ++s) {
    for (int k = 0; k < 5; ++k) {
      int rc = g->elem == 4 ? stage_impl<float>(g, k, dt, st) : stage_impl<double>(g, k, dt, st);
      if (rc) return rc;
    }
    g->t += dt;
    if (g->rec_n > 0) {
      cudaError_t e = g->elem == 4
                          ? sbp::launch_receivers<float>((const float*)g->q[g->cur], g->dims, g->rec_off, g->rec_n,
                                                         g->nb, 9 * g->dims.fs, (float*)g->traces, g->n_t, g->step,
                                                         st)
                          : sbp::launch_receivers<double>((const double*)g->q[g->cur], g->dims, g->rec_off,
                                                          g->rec_n, g->nb, 9 * g->dims.fs, (double*)g->traces,
                                                          g->n_t, g->step, st);
      if (e != cudaSuccess) return cuda_fail(e, "receivers");
    }
    ++g->step;
  }
  return SBP_OK;
}

int sbp_set_kernel_path(SbpGrid* g, int32_t path) {
  if (!g) return fail(SBP_ERR_ARG, "null grid");
  if (path != 0 && path != 1) return fail(SBP_ERR_ARG, "kernel path must be 0 or 1");
  g->use_tiled = path == 0;
  return SBP_OK;
}

int sbp_kernel_timing(SbpGrid* g, int32_t enable) {
  if (!g) return fail(SBP_ERR_ARG, "null grid");
  g->timing = enable != 0;
  return SBP_OK;
}

int sbp_kernel_times(SbpGrid* g, double* ms, int64_t* launches) {
  if (!g || !ms || !launches) return fail(SBP_ERR_ARG, "null argument");
  for (int k = 0; k < 3; ++k) {
    ms[k] = 0.0;
    launches[k] = 0;
  }
  for (auto& p : g->ev_pending) {
    cudaError_t e = cudaEventSynchronize(p.second.second);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, p.second.first, p.second.second);
    if (e != cudaSuccess) return cuda_fail(e, "kernel timing events");
    ms[p.first] += t;
    launches[p.first] += 1;
    g->ev_pool.push_back(p.second.first);
    g->ev_pool.push_back(p.second.second);
  }
  g->ev_pending.clear();
  return SBP_OK;
}

int sbp_current(const SbpGrid* g, int32_t* which) {
  if (!g || !which) return fail(SBP_ERR_ARG, "null argument");
  *which = g->cur;
  return SBP_OK;
}

int sbp_set_time(SbpGrid* g, double t, int64_t step) {
  if (!g) return fail(SBP_ERR_ARG, "null grid");
  if (step < 0) return fail(SBP_ERR_ARG, "negative step counter");
  if (!isfinite(t)) return fail(SBP_ERR_ARG, "time must be finite");
  g->t = t;
  g->step = step;
  return SBP_OK;
}

int sbp_get_time(const SbpGrid* g, double* t, int64_t* step) {
  if (!g) return fail(SBP_ERR_ARG, "null grid");
  if (t) *t = g->t;
  if (step) *step = g->step;
  return SBP_OK;
}

int sbp_energy(SbpGrid* g, double* out, void* stream) {
  if (int rc = check_ready(g)) return rc;
  if (!g->material) return fail(SBP_ERR_STATE, "material not set (sbp_set_material)");
  if (!out) return fail(SBP_ERR_ARG, "null output");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = g->elem == 4 ? sbp::launch_energy<float>((const float*)g->q[g->cur], (const float*)g->mat,
                                                           g->dims, g->desc.order, g->partial, sbp::energy_blocks(),
                                                           g->eout, g->status, st, g->slab)
                               : sbp::launch_energy<double>((const double*)g->q[g->cur], (const double*)g->mat,
                                                            g->dims, g->desc.order, g->partial,
                                                            sbp::energy_blocks(), g->eout, g->status, st, g->slab);
  if (e != cudaSuccess) return cuda_fail(e, "energy");
  double v = 0.0;
  e = cudaMemcpyAsync(&v, g->eout, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "energy readback");
  *out = v;
  if (!isfinite(v)) return fail(SBP_ERR_NONFINITE, "energy is not finite");
  return SBP_OK;
}

int sbp_set_sources(SbpGrid* g, int32_t n, const SbpSource* srcs, const double* jmet, void* stream) {
  if (int rc = check_ready(g)) return rc;
  if (g->slab.ns_global > 0 && n > 0) return fail(SBP_ERR_UNSUPPORTED, "point sources on slab grids are not built");
  if (n == 0 || !srcs) {
    g->src_n = 0;
    return SBP_OK;
  }
  if (n < 0 || n > g->nb) return fail(SBP_ERR_ARG, "at most one source per bound state (%d states)", g->nb);
  if (!jmet) return fail(SBP_ERR_ARG, "set_source needs the FP64 Jacobian (jmet)");
  for (int m = 0; m < n; ++m) {
    const SbpSource* src = &srcs[m];
    for (int a = 0; a < 3; ++a)
      if (!(src->ref[a] >= 0.0 && src->ref[a] <= 1.0)) return fail(SBP_ERR_ARG, "source outside the reference cube");
    if (src->stf != 0 && src->stf != 1) return fail(SBP_ERR_ARG, "unknown source time function");
    if (src->stf != srcs[0].stf || src->f0 != srcs[0].f0 || src->t0 != srcs[0].t0 || src->T != srcs[0].T)
      return fail(SBP_ERR_UNSUPPORTED, "sources of one batch must share their time function");
  }
  const int order = g->desc.order;
  const int mo = op_info(order).accuracy + 1;
  const int N[3] = {g->desc.nq, g->desc.nr, g->desc.ns};
  const int n1 = mo + 1, per = n1 * n1 * n1;
  std::vector<long long> off((size_t)per * n);
  std::vector<double> w((size_t)per * n * 6);
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaStreamSynchronize(st);
  auto wgt = [&](int a, int pos) { return norm_weight_any(order, pos, N[a]) / (N[a] - 1); };
  for (int m = 0; m < n && e == cudaSuccess; ++m) {
    const SbpSource* src = &srcs[m];
    int start[3];
    double phi[3][10];  // up to accuracy + 2 = 9 nodes per axis
    for (int a = 0; a < 3; ++a) sbp::delta_1d(src->ref[a], N[a], mo, &start[a], phi[a]);
    double Jrow[10];
    for (int kk = 0, c = 0; kk < n1; ++kk)
      for (int jj = 0; jj < n1; ++jj) {
        // the Jacobian along this q row of the source's stencil box, one copy per row
        const long long row = (long long)(start[2] + kk) * g->dims.plane + (long long)(start[1] + jj) * g->dims.ldq +
                              start[0];
        if (e == cudaSuccess) e = cudaMemcpy(Jrow, jmet + row, sizeof(double) * n1, cudaMemcpyDeviceToHost);
        for (int ii = 0; ii < n1; ++ii, ++c) {
          const long long node = row + ii;
          const double J = Jrow[ii];
          const double H = wgt(0, start[0] + ii) * wgt(1, start[1] + jj) * wgt(2, start[2] + kk);
          const double delta = phi[0][ii] * phi[1][jj] * phi[2][kk] / (J * H);
          const size_t idx = (size_t)m * per + c;
          off[idx] = (long long)m * 9 * g->dims.fs + node;
          for (int q = 0; q < 6; ++q) w[idx * 6 + q] = -src->moment[q] * delta;
        }
      }
  }
  if (e != cudaSuccess) return cuda_fail(e, "source Jacobian readback");
  cudaFree(g->src_off);
  cudaFree(g->src_w);
  g->src_off = nullptr;
  g->src_w = nullptr;
  const size_t nn = (size_t)per * n;
  e = cudaMalloc(&g->src_off, sizeof(long long) * nn);
  if (e == cudaSuccess) e = cudaMalloc(&g->src_w, sizeof(double) * nn * 6);
  if (e == cudaSuccess) e = cudaMemcpy(g->src_off, off.data(), sizeof(long long) * nn, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(g->src_w, w.data(), sizeof(double) * nn * 6, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "source buffers");
  g->src = srcs[0];
  g->src_n = (int)nn;
  return SBP_OK;
}

int sbp_set_source(SbpGrid* g, const SbpSource* src, const double* jmet, void* stream) {
  return sbp_set_sources(g, src ? 1 : 0, src, jmet, stream);
}

int sbp_set_slab(SbpGrid* g, int32_t ns_global, int32_t k_offset, int32_t ghost_lo, int32_t ghost_hi) {
  if (!g) return fail(SBP_ERR_ARG, "null grid");
  if (g->bound) return fail(SBP_ERR_STATE, "sbp_set_slab must come before sbp_bind");
  const OpInfo I = op_info(g->desc.order);
  const int L = g->desc.ns;
  int32_t nmin = 0;
  sbp_min_nodes(g->desc.order, &nmin);
  if (ns_global < nmin) return fail(SBP_ERR_ARG, "the block needs at least %d planes", nmin);
  if (ghost_lo < 0 || ghost_hi < 0 || (ghost_lo > 0 && ghost_lo < I.reach) || (ghost_hi > 0 && ghost_hi < I.reach))
    return fail(SBP_ERR_ARG, "ghost planes: 0 (a face of the block) or at least %d", I.reach);
  if (L - ghost_lo - ghost_hi < 1) return fail(SBP_ERR_ARG, "the slab owns no plane");
  if (k_offset < 0 || k_offset + L > ns_global) return fail(SBP_ERR_ARG, "slab planes outside the block");
  if ((ghost_lo == 0) != (k_offset == 0) || (ghost_hi == 0) != (k_offset + L == ns_global))
    return fail(SBP_ERR_ARG, "ghost planes must be 0 exactly at the block's faces");
  const int cw = 2 * I.b + I.reach;  // closure rows reach at most this many planes from a face
  if ((ghost_lo == 0 || ghost_hi == 0) && L < cw)
    return fail(SBP_ERR_ARG, "a slab at a face of the block needs at least %d local planes", cw);
  if (ghost_lo == 0 && ghost_hi == 0) {  // the whole block: no decomposition
    g->slab = sbp::SlabS{};
    return SBP_OK;
  }
  g->slab.ghost_lo = ghost_lo;
  g->slab.ghost_hi = ghost_hi;
  g->slab.k_offset = k_offset;
  g->slab.ns_global = ns_global;
  return SBP_OK;
}

int sbp_set_interface(SbpGrid* g, int32_t face, const void* other_trace) {
  if (!g) return fail(SBP_ERR_ARG, "null grid");
  if (face < 0 || face > 5) return fail(SBP_ERR_ARG, "face must be 0..5");
  if (g->desc.bc_kind[face] != SBP_BC_INTERFACE) return fail(SBP_ERR_ARG, "face %d is not an interface face", face);
  g->iface[face] = other_trace;
  return SBP_OK;
}

int sbp_interface_trace(SbpGrid* g, int32_t face, const void* q, void* trace, void* stream) {
  if (int rc = check_ready(g)) return rc;
  if (!g->material) return fail(SBP_ERR_STATE, "material not set (sbp_set_material)");
  if (face < 0 || face > 5) return fail(SBP_ERR_ARG, "face must be 0..5");
  if (!trace) return fail(SBP_ERR_ARG, "null trace buffer");
  const void* src = q ? q : g->q[g->cur];
  const long long bs = 9 * g->dims.fs;
  cudaError_t e = g->elem == 4 ? sbp::launch_interface_trace<float>((const float*)src, (const float*)g->met,
                                                                    (const float*)g->mat, g->dims, face, g->nb, bs,
                                                                    (float*)trace, (cudaStream_t)stream)
                               : sbp::launch_interface_trace<double>((const double*)src, (const double*)g->met,
                                                                     (const double*)g->mat, g->dims, face, g->nb, bs,
                                                                     (double*)trace, (cudaStream_t)stream);
  return e == cudaSuccess ? SBP_OK : cuda_fail(e, "interface trace");
}

int sbp_probe_fp64_rate(int32_t iters, double* tflops, void* stream) {
  if (!tflops || iters < 1000 || iters > 100000000) return fail(SBP_ERR_ARG, "iters must lie in 1000..1e8");
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(e, "device query");
  const int blocks = sms * 8;  // 2048 threads per SM: full occupancy
  double* sink = nullptr;
  e = cudaMalloc(&sink, sizeof(double) * blocks);
  float ms = 0.f;
  if (e == cudaSuccess) e = sbp::probe_fp64_fma(iters, blocks, sink, &ms, (cudaStream_t)stream);
  cudaFree(sink);
  if (e != cudaSuccess) return cuda_fail(e, "FP64 rate probe");
  *tflops = 16.0 * iters * blocks * 256.0 / (ms * 1e-3) / 1e12;
  return SBP_OK;
}

int sbp_set_batch(SbpGrid* g, int32_t nb) {
  if (!g) return fail(SBP_ERR_ARG, "null grid");
  if (g->bound) return fail(SBP_ERR_STATE, "sbp_set_batch must come before sbp_bind");
  if (nb < 1 || nb > 1024) return fail(SBP_ERR_ARG, "batch must lie in 1..1024");
  g->nb = nb;
  return SBP_OK;
}

int sbp_set_receivers(SbpGrid* g, int32_t n, const int32_t* ijk, void* traces, int32_t n_t) {
  if (int rc = check_ready(g)) return rc;
  if (n < 0 || (n > 0 && (!ijk || n_t <= 0))) return fail(SBP_ERR_ARG, "bad receiver arguments");
  if (n > 65535) return fail(SBP_ERR_ARG, "at most 65535 receivers");
  // validate every receiver before the current ones are dropped
  std::vector<int32_t> off(n);
  for (int r = 0; r < n; ++r) {
    const int i = ijk[3 * r], j = ijk[3 * r + 1], k = ijk[3 * r + 2];
    if (i < 0 || i >= g->desc.nq || j < 0 || j >= g->desc.nr || k < 0 || k >= g->desc.ns)
      return fail(SBP_ERR_ARG, "receiver %d outside the grid", r);
    off[r] = (int32_t)((long long)k * g->dims.plane + (long long)j * g->dims.ldq + i);
  }
  const size_t trace_bytes = (size_t)g->nb * n * 3 * (size_t)(n > 0 ? n_t : 0) * g->elem;
  void* own = nullptr;
  if (n > 0 && !traces) {
    // the library keeps the traces; sbp_record_receivers copies them out
    cudaError_t e = cudaMalloc(&own, trace_bytes);
    if (e == cudaSuccess) e = cudaMemset(own, 0, trace_bytes);
    if (e != cudaSuccess) {
      cudaFree(own);
      return cuda_fail(e, "trace buffer");
    }
  }
  cudaFree(g->rec_off);
  if (g->traces_owned) cudaFree(g->traces);
  g->rec_off = nullptr;
  g->traces = nullptr;
  g->traces_owned = false;
  g->rec_n = 0;
  g->n_t = 0;
  if (n == 0) return SBP_OK;
  cudaError_t e = cudaMalloc(&g->rec_off, sizeof(int32_t) * n);
  if (e == cudaSuccess) e = cudaMemcpy(g->rec_off, off.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(own);
    return cuda_fail(e, "receiver buffers");
  }
  g->rec_n = n;
  g->traces = own ? own : traces;
  g->traces_owned = own != nullptr;
  g->n_t = n_t;
  return SBP_OK;
}

int sbp_set_receivers_xyz(SbpGrid* g, int32_t n, const double* xyz, const double* coords, int32_t face,
                          void* traces, int32_t n_t, int32_t* ijk_out) {
  if (int rc = check_ready(g)) return rc;
  if (n < 0 || n > 65535) return fail(SBP_ERR_ARG, "receiver count must lie in 0..65535");
  if (n == 0) return sbp_set_receivers(g, 0, nullptr, nullptr, 0);
  if (!xyz || !coords || n_t <= 0) return fail(SBP_ERR_ARG, "bad receiver arguments");
  if (face < -1 || face > 5) return fail(SBP_ERR_ARG, "face must be -1 (every node) or 0..5");
  for (int r = 0; r < 3 * n; ++r)
    if (!isfinite(xyz[r])) return fail(SBP_ERR_ARG, "receiver %d: position is not finite", r / 3);
  double* tg = nullptr;
  unsigned long long* scratch = nullptr;
  cudaError_t e = cudaMalloc(&tg, sizeof(double) * 3 * n);
  if (e == cudaSuccess) e = cudaMalloc(&scratch, sizeof(unsigned long long) * 2 * n);
  if (e == cudaSuccess) e = cudaMemcpy(tg, xyz, sizeof(double) * 3 * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = sbp::launch_locate(coords, g->dims, face, tg, n, scratch, scratch + n, nullptr);
  std::vector<unsigned long long> node(n);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess)
    e = cudaMemcpy(node.data(), scratch + n, sizeof(unsigned long long) * n, cudaMemcpyDeviceToHost);
  cudaFree(tg);
  cudaFree(scratch);
  if (e != cudaSuccess) return cuda_fail(e, "receiver location");
  std::vector<int32_t> ijk(3 * n);
  const long long nq = g->desc.nq, nr = g->desc.nr;
  for (int r = 0; r < n; ++r) {
    if (node[r] == ~0ULL) return fail(SBP_ERR_ARG, "receiver %d: no node at a finite distance", r);
    const long long t = (long long)node[r];
    ijk[3 * r] = (int32_t)(t % nq);
    ijk[3 * r + 1] = (int32_t)((t / nq) % nr);
    ijk[3 * r + 2] = (int32_t)(t / (nq * nr));
  }
  if (int rc = sbp_set_receivers(g, n, ijk.data(), traces, n_t)) return rc;
  if (ijk_out) memcpy(ijk_out, ijk.data(), sizeof(int32_t) * 3 * n);
  return SBP_OK;
}

int sbp_record_receivers(SbpGrid* g, void* dst, int32_t flags, void* stream) {
  if (int rc = check_ready(g)) return rc;
  if (g->rec_n == 0) return fail(SBP_ERR_STATE, "no receivers set (sbp_set_receivers)");
  if (!dst) return fail(SBP_ERR_ARG, "null destination");
  if (flags & ~SBP_MEM_HOST) return fail(SBP_ERR_ARG, "flags: only SBP_MEM_HOST applies to traces");
  const size_t bytes = (size_t)g->nb * g->rec_n * 3 * (size_t)g->n_t * g->elem;
  cudaStream_t st = (cudaStream_t)stream;
  const bool host = (flags & SBP_MEM_HOST) != 0;
  cudaError_t e = cudaMemcpyAsync(dst, g->traces, bytes, host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && host) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? SBP_OK : cuda_fail(e, "trace copy");
}

int sbp_set_state(SbpGrid* g, const void* src, int32_t flags, void* stream) {
  if (int rc = check_ready(g)) return rc;
  if (!src) return fail(SBP_ERR_ARG, "null source");
  if (flags & ~(SBP_MEM_HOST | SBP_LAYOUT_DENSE)) return fail(SBP_ERR_ARG, "unknown flags");
  return copy_state(g, g->q[g->cur], src, flags, true, (cudaStream_t)stream);
}

int sbp_get_state(SbpGrid* g, void* dst, int32_t flags, void* stream) {
  if (int rc = check_ready(g)) return rc;
  if (!dst) return fail(SBP_ERR_ARG, "null destination");
  if (flags & ~(SBP_MEM_HOST | SBP_LAYOUT_DENSE | SBP_MEM_ASYNC)) return fail(SBP_ERR_ARG, "unknown flags");
  return copy_state(g, g->q[g->cur], dst, flags, false, (cudaStream_t)stream);
}

int sbp_rhs_adjoint(SbpGrid* g, const void* w, void* out, void* scratch, void* stream) {
  if (int rc = check_ready(g)) return rc;
  if (has_interface(g)) return fail(SBP_ERR_UNSUPPORTED, "the adjoint with interface faces is not built");
  if (g->slab.ns_global > 0) return fail(SBP_ERR_UNSUPPORTED, "the adjoint on slab grids is not built");
  if (!op_info(g->desc.order).adjoint) return fail(SBP_ERR_UNSUPPORTED, "the adjoint is built for orders 2, 4, 6");
  if (!g->material) return fail(SBP_ERR_STATE, "material not set (sbp_set_material)");
  if (!w || !out || !scratch || w == out || w == scratch || out == scratch)
    return fail(SBP_ERR_ARG, "rhs_adjoint needs distinct input, output and scratch buffers");
  return g->elem == 4 ? adjoint_impl<float>(g, 0, 0, 0.0, nullptr, out, w, nullptr, scratch, nullptr, nullptr,
                                            (cudaStream_t)stream)
                      : adjoint_impl<double>(g, 0, 0, 0.0, nullptr, out, w, nullptr, scratch, nullptr, nullptr,
                                             (cudaStream_t)stream);
}

int sbp_adjoint_stage(SbpGrid* g, int32_t stage, double dt, const void* u_stage, void* ubar, void* wbar,
                      void* scratch, const double* rlmj, double* grad, void* stream) {
  if (int rc = check_ready(g)) return rc;
  if (!op_info(g->desc.order).adjoint) return fail(SBP_ERR_UNSUPPORTED, "the adjoint is built for orders 2, 4, 6");
  if (g->slab.ns_global > 0) return fail(SBP_ERR_UNSUPPORTED, "the adjoint on slab grids is not built");
  if (has_interface(g)) return fail(SBP_ERR_UNSUPPORTED, "the adjoint with interface faces is not built");
  if (!g->material) return fail(SBP_ERR_STATE, "material not set (sbp_set_material)");
  if (stage < 0 || stage > 4) return fail(SBP_ERR_ARG, "stage must be 0..4");
  if (!(dt > 0) || !isfinite(dt)) return fail(SBP_ERR_ARG, "dt must be positive and finite");
  if (!ubar || !wbar || !scratch) return fail(SBP_ERR_ARG, "null adjoint buffer");
  if (grad && (!u_stage || !rlmj)) return fail(SBP_ERR_ARG, "the gradient needs the stage state and rho, lambda, mu, J");
  return g->elem == 4 ? adjoint_impl<float>(g, 1, stage, dt, u_stage, ubar, wbar, wbar, scratch, rlmj, grad,
                                            (cudaStream_t)stream)
                      : adjoint_impl<double>(g, 1, stage, dt, u_stage, ubar, wbar, wbar, scratch, rlmj, grad,
                                             (cudaStream_t)stream);
}

int sbp_adjoint_step(SbpGrid* g, double dt, const void* u_stages, void* ubar, void* wbar, void* scratch,
                     const double* rlmj, double* grad, void* stream) {
  if (int rc = check_ready(g)) return rc;
  if (!op_info(g->desc.order).adjoint) return fail(SBP_ERR_UNSUPPORTED, "the adjoint is built for orders 2, 4, 6");
  if (g->slab.ns_global > 0) return fail(SBP_ERR_UNSUPPORTED, "the adjoint on slab grids is not built");
  if (has_interface(g)) return fail(SBP_ERR_UNSUPPORTED, "the adjoint with interface faces is not built");
  if (!g->material) return fail(SBP_ERR_STATE, "material not set (sbp_set_material)");
  if (!(dt > 0) || !isfinite(dt)) return fail(SBP_ERR_ARG, "dt must be positive and finite");
  if (!ubar || !wbar || !scratch) return fail(SBP_ERR_ARG, "null adjoint buffer");
  if (grad && (!u_stages || !rlmj)) return fail(SBP_ERR_ARG, "the gradient needs the stage states and rho, lambda, mu, J");
  cudaStream_t st = (cudaStream_t)stream;
  if (!g->use_tiled) {
    // the general kernels: the five stages one by one
    const long long grp = 9LL * g->nb * g->dims.fs * g->elem;  // bytes of one group of B states
    for (int k = 4; k >= 0; --k) {
      const void* uk = u_stages ? (const char*)u_stages + k * grp : nullptr;
      const int rc = g->elem == 4 ? adjoint_impl<float>(g, 1, k, dt, uk, ubar, wbar, wbar, scratch, rlmj, grad, st)
                                  : adjoint_impl<double>(g, 1, k, dt, uk, ubar, wbar, wbar, scratch, rlmj, grad, st);
      if (rc) return rc;
    }
    return SBP_OK;
  }
  return g->elem == 4 ? adjoint_step_impl<float>(g, dt, u_stages, ubar, wbar, scratch, rlmj, grad, st)
                      : adjoint_step_impl<double>(g, dt, u_stages, ubar, wbar, scratch, rlmj, grad, st);
}

int sbp_misfit(SbpGrid* g, const void* q, const double* data, double weight, double* acc, void* ubar, void* stream) {
  if (int rc = check_ready(g)) return rc;
  if (g->rec_n == 0) return fail(SBP_ERR_STATE, "no receivers set (sbp_set_receivers)");
  if (!q || !data) return fail(SBP_ERR_ARG, "null state or data");
  const long long bs = 9 * g->dims.fs;
  cudaError_t e = g->elem == 4 ? sbp::launch_misfit<float>((const float*)q, g->dims, g->rec_off, g->rec_n, g->nb, bs,
                                                            data, weight, acc, (float*)ubar, (cudaStream_t)stream)
                               : sbp::launch_misfit<double>((const double*)q, g->dims, g->rec_off, g->rec_n, g->nb,
                                                             bs, data, weight, acc, (double*)ubar,
                                                             (cudaStream_t)stream);
  return e == cudaSuccess ? SBP_OK : cuda_fail(e, "misfit");
}

int sbp_selftest_wait_timeout(SbpGrid* g, uint32_t polls, void* stream) {
  if (int rc = check_ready(g)) return rc;
  if (polls == 0 || polls > (1u << 20)) return fail(SBP_ERR_ARG, "polls must lie in 1..2^20");
  cudaError_t e = sbp::launch_wait_selftest(polls, g->status, (cudaStream_t)stream);
  return e == cudaSuccess ? SBP_OK : cuda_fail(e, "wait self-test");
}

int sbp_status(SbpGrid* g, uint32_t* bits, void* stream) {
  if (int rc = check_ready(g)) return rc;
  if (!bits) return fail(SBP_ERR_ARG, "null output");
  cudaStream_t st = (cudaStream_t)stream;
  unsigned v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, g->status, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->status, 0, sizeof(unsigned), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "status readback");
  *bits = v;
  return SBP_OK;
}

}  // extern "C"
