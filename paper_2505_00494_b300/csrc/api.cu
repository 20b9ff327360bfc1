// C ABI of the QR-CTMRG library (declared in include/qrctm.h).
//
// The context never allocates device memory: every buffer is a region of
// the caller's workspace, laid out by make_plan().  Errors are reported as
// status codes plus a per-context message; kernel-side failures raise bits
// of a device error word that the host reads at every synchronisation.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include <nvtx3/nvToolsExt.h>

#include "ctx.cuh"
#include "tc_gemm.cuh"
#include "grad.cuh"

using namespace qrctm;

namespace {

inline size_t al(size_t x) { return (x + 255) & ~size_t(255); }

bool cfg_valid(const qrctm_config& c) {
  if (c.d < 1 || c.D < 1 || c.chi < 1 || c.chi > 1024) return false;
  if (c.precision != QRCTM_FP64 && c.precision != QRCTM_SPLIT) return false;
  if (c.layers < 0 || c.layers > 3) return false;
  if (c.check_every < 0 || c.warmup_steps < -1) return false;
  const bool net = c.layers == QRCTM_LAYERS_NETWORK;
  if (net && (c.d != 1 || c.precision != QRCTM_FP64 || c.with_grad || c.with_nnn)) return false;
  if (c.opt_history < 0 || c.opt_history > 32) return false;
  if (c.opt_history > 0 && !c.with_grad) return false;
  if (c.grad_store < 0 || c.grad_store > kGradMaxUnroll) return false;
  if (c.grad_store > 0 && !c.with_grad) return false;
  const long long D2 = net ? (long long)c.D : (long long)c.D * c.D;
  if (D2 > 4096 || (long long)c.chi * D2 > (1ll << 20)) return false;
  if (c.chi < D2) return false;
  if (c.precision == QRCTM_SPLIT && c.D < 2) return false;
  if (c.method != QRCTM_METHOD_QR && c.method != QRCTM_METHOD_EIGEN) return false;
  if (c.method == QRCTM_METHOD_EIGEN && c.precision != QRCTM_FP64) return false;
  return true;
}

qrctm_status set_err(qrctm_ctx* c, qrctm_status s, const char* msg) {
  if (c) c->last_error = msg;
  return s;
}

qrctm_status cuda_fail(qrctm_ctx* c, cudaError_t e, const char* where) {
  if (c) {
    char buf[256];
    snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
    c->last_error = buf;
  }
  return QRCTM_ERR_CUDA;
}

// Synchronise the stream and translate the device error word.
qrctm_status sync_check(qrctm_ctx* c, const char* where) {
  // one wait: a device-to-host copy into pageable memory returns once the
  // stream's earlier work and the copy are done (and reports their errors)
  int flag = 0;
  cudaError_t e = cudaMemcpyAsync(&flag, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) return cuda_fail(c, e, where);
  if (flag) {
    cudaMemsetAsync(c->err, 0, sizeof(int), c->st);
    // an abandoned wait can leave the QR arrival counter non-zero
    if (flag & ERRF_TIMEOUT) cudaMemsetAsync(c->qrw.bar, 0, sizeof(GridBar), c->st);
    cudaStreamSynchronize(c->st);
    if (flag & ERRF_TIMEOUT) return set_err(c, QRCTM_ERR_TIMEOUT, "device wait timed out");
    if (flag & ERRF_NUMERIC) return set_err(c, QRCTM_ERR_NUMERIC, "NaN/Inf or zero norm");
    return set_err(c, QRCTM_ERR_NUMERIC, "device size check failed");
  }
  return QRCTM_OK;
}

}  // namespace

namespace qrctm {

void panel_hook(void* user, int begin);

// Regions in a fixed order; the same function sizes and carves.
size_t make_plan(const qrctm_config& cfg, bool carve, qrctm_ctx* c) {
  const bool net = cfg.layers == QRCTM_LAYERS_NETWORK;
  const size_t d = cfg.d, D = cfg.D, D2 = net ? D : D * D, chi = cfg.chi, m = chi * D2;
  const bool split = (cfg.layers == QRCTM_LAYERS_SPLIT) ||
                     (cfg.layers == QRCTM_LAYERS_AUTO && 2 * d < D2);
  size_t off = 0;
  auto take = [&](double** dst, size_t n_doubles) {
    size_t o = off;
    off += al(sizeof(double) * (n_doubles > 0 ? n_doubles : 1));
    if (carve && dst) *dst = reinterpret_cast<double*>(c->ws + o);
  };
  auto P = [&](double*& ref) { return carve ? &ref : nullptr; };
  static double* dummy;
  qrctm_ctx* cc = carve ? c : nullptr;
#define R_(field) P(cc ? cc->field : dummy)
  // network mode: A and tmpA hold the network tensor (D2^4 doubles)
  const size_t nA = net ? D2 * D2 * D2 * D2 : d * D2 * D2, nC = chi * chi, nT = chi * D2 * chi;
  take(R_(A), nA);
  take(R_(tmpA), nA);
  take(R_(C), nC);
  take(R_(T), nT);
  take(R_(Cn), nC);
  take(R_(Tn), nT);
  take(R_(Craw), nC);
  take(R_(Traw), nT);
  take(R_(Mcm), m * chi);
  take(R_(Q), m * chi);
  take(R_(R), nC);
  take(R_(X1), m * m);
  take(R_(Z), m * m * d);
  take(R_(X2), m * m);
  take(R_(Y2), m * chi);
  take(R_(Xs), m * chi);
  take(R_(Yw), m * chi);
  take(R_(spec_work), nC + 8 * chi + 16);
  take(R_(spec_work2), nC + 8 * chi + 16);
  take(R_(C_init), nC);
  take(R_(s_cur), chi);
  take(R_(s_prev), chi);
  take(R_(delta_d), 8);
  take(R_(partials), std::max<size_t>(1024, (size_t)16 * kTraceParts));
  take(R_(a), split ? 1 : D2 * D2 * D2 * D2);
  // energy patches (iPEPS only)
  take(R_(E1), net ? 1 : d * d * m * m);
  take(R_(E2), net ? 1 : d * d * m * chi);
  if (cfg.with_nnn) take(R_(E3), d * d * m * m);
  else if (carve) c->E3 = nullptr;
  take(R_(rho), 64);
  take(R_(e_d), 8);
#undef R_
  // split precision buffers (floats; carved as double regions of half size)
  if (cfg.precision == QRCTM_SPLIT) {
    auto p4 = [](size_t x) { return (x + 3) & ~size_t(3); };
    const size_t chp = p4(chi), mp = p4(m), D2p = p4(D2), dD2p = p4(d * D2);
    auto takef = [&](float** dst, size_t n_floats) {
      size_t o = off;
      off += al(sizeof(float) * (n_floats > 0 ? n_floats : 1));
      if (carve) *dst = reinterpret_cast<float*>(c->ws + o);
    };
    static float* fdummy;
    takef(carve ? &c->T32 : &fdummy, m * chp);
    takef(carve ? &c->C32 : &fdummy, chi * chp);
    takef(carve ? &c->Qt32 : &fdummy, m * chp);
    takef(carve ? &c->Qc32 : &fdummy, chi * mp);
    takef(carve ? &c->T32lo : &fdummy, m * chp);
    takef(carve ? &c->C32lo : &fdummy, chi * chp);
    takef(carve ? &c->Qt32lo : &fdummy, m * chp);
    takef(carve ? &c->Qc32lo : &fdummy, chi * mp);
    takef(carve ? &c->Rt32lo : &fdummy, chi * chp);
    takef(carve ? &c->Ts32 : &fdummy, m * chp);
    takef(carve ? &c->Rt32 : &fdummy, chi * chp);
    takef(carve ? &c->Aket32 : &fdummy, d * D2 * D2p);
    takef(carve ? &c->Abra32 : &fdummy, D2 * dD2p);
    const size_t part = size_t(1) << 24;
    takef(carve ? &c->tc_part : &fdummy, part);
    takef(carve ? &c->qr32 : &fdummy, qr_split_floats((int)m, (int)chi));
    if (carve) c->tc_part_elems = (long long)part;
    // the FP32 intermediates X1, Z, X2, Y2 reuse the FP64 regions of the same
    // names: for D >= 2 each needs at most as many bytes as its FP64 region
  } else if (carve) {
    c->T32 = c->C32 = c->Qt32 = c->Qc32 = c->Ts32 = c->Rt32 = c->Aket32 = c->Abra32 = nullptr;
    c->T32lo = c->C32lo = c->Qt32lo = c->Qc32lo = c->Rt32lo = nullptr;
    c->qr32 = nullptr;
    c->tc_part = nullptr;
    c->tc_part_elems = 0;
  }
  {
    size_t o = off;
    off += al(qr_work_bytes((int)m, (int)chi));
    if (carve) {
      c->qrw = qr_carve(c->ws + o, (int)m, (int)chi);
      c->qrw.hook = panel_hook;
      c->qrw.hook_user = c;
    }
  }
  {
    size_t o = off;
    off += 256;
    if (carve) c->err = reinterpret_cast<int*>(c->ws + o);
  }
  if (cfg.with_grad) {
    size_t gb = grad_bytes((int)d, (int)D, (int)chi);
    size_t o = off;
    off += al(gb);
    if (carve) { c->G = c->ws + o; c->G_bytes = gb; }
    // tapes of the unrolled gradient's steps
    const size_t tb = tape_bytes((int)d, (int)D, (int)chi), ts = tb * (size_t)cfg.grad_store;
    o = off;
    off += al(ts);
    if (carve) {
      c->tape_store = cfg.grad_store > 0 ? c->ws + o : nullptr;
      c->tape_store_k = cfg.grad_store;
    }
  } else if (carve) {
    c->G = nullptr; c->G_bytes = 0;
    c->tape_store = nullptr; c->tape_store_k = 0;
  }
  // FP32 operand copies for the split-precision energy and adjoint
  // contractions: the energy's largest pairs a d^2-batched (chi D^2)^2
  // operand with an unbatched one ((d^2 + 1) (chi D^2)^2 floats); with the J2
  // gradient, the adjoint of the 2x2-patch product reads two operands of
  // d^2 (chi D^2)^2 each, which must also fit here to run on the tensor cores
  if (cfg.precision == QRCTM_SPLIT) {
    const size_t mm = m * m;
    const size_t per = (cfg.with_grad && cfg.with_nnn) ? 2 * d * d + 2 : d * d + 2;
    const size_t floats = per * mm + (size_t(1) << 20);
    size_t o = off;
    off += al(sizeof(float) * floats);
    if (carve) { c->mm32 = reinterpret_cast<float*>(c->ws + o); c->mm32_floats = floats; }
  } else if (carve) {
    c->mm32 = nullptr; c->mm32_floats = 0;
  }
  // L-BFGS optimisation buffers
  if (cfg.opt_history > 0) {
    const size_t h = cfg.opt_history, n = d * D2 * D2;
    take(carve ? &c->opt_S : nullptr, h * n);
    take(carve ? &c->opt_Y : nullptr, h * n);
    take(carve ? &c->opt_x : nullptr, n);
    take(carve ? &c->opt_xt : nullptr, n);
    take(carve ? &c->opt_g : nullptr, n);
    take(carve ? &c->opt_gt : nullptr, n);
    take(carve ? &c->opt_p : nullptr, n);
    take(carve ? &c->opt_q : nullptr, n);
    take(carve ? &c->opt_out : nullptr, 16);
    take(carve ? &c->opt_Cp : nullptr, nC);
    take(carve ? &c->opt_Tp : nullptr, nT);
    take(carve ? &c->opt_Cc : nullptr, nC);
    take(carve ? &c->opt_Tc : nullptr, nT);
    if (carve) c->opt_hist = (int)h;
  } else if (carve) {
    c->opt_hist = 0;
    c->opt_S = c->opt_Y = c->opt_x = c->opt_xt = c->opt_g = c->opt_gt = c->opt_p = c->opt_q =
        c->opt_out = c->opt_Cp = c->opt_Tp = c->opt_Cc = c->opt_Tc = nullptr;
  }
  // standard method: dense enlarged corner, eigenvalues, solver workspace
  if (cfg.method == QRCTM_METHOD_EIGEN) {
    const size_t ew = eigen_work_doubles((long long)m);
    size_t o = off;
    off += al(sizeof(double) * m * m);
    if (carve) c->eig_E = reinterpret_cast<double*>(c->ws + o);
    o = off; off += al(sizeof(double) * m);
    if (carve) c->eig_w = reinterpret_cast<double*>(c->ws + o);
    o = off; off += al(sizeof(double) * ew);
    if (carve) { c->eig_work = reinterpret_cast<double*>(c->ws + o); c->eig_work_doubles = ew; }
    o = off; off += al(sizeof(int) * (chi + 64));
    if (carve) { c->eig_info = reinterpret_cast<int*>(c->ws + o); c->eig_idx = c->eig_info + 64; }
  } else if (carve) {
    c->eig_E = c->eig_w = c->eig_work = nullptr;
    c->eig_work_doubles = 0;
    c->eig_info = c->eig_idx = nullptr;
  }
  if (carve) {
    c->grad_keep_env = false;
    c->network = net;
    c->split_layers = split;
    c->mm_split = false;   // set for the duration of a split-precision gradient
    c->solver = nullptr;
  }
  return off;
}

cudaEvent_t phase_begin(qrctm_ctx* c) {
  if (!c->prof) return nullptr;
  if (c->ev_pool.empty()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    c->ev_pool.push_back(e);
  }
  cudaEvent_t a = c->ev_pool.back();
  c->ev_pool.pop_back();
  cudaEventRecord(a, c->st);
  return a;
}

void phase_end(qrctm_ctx* c, int ph, cudaEvent_t a) {
  if (!a) return;
  cudaEvent_t b;
  if (c->ev_pool.empty()) {
    if (cudaEventCreate(&b) != cudaSuccess) { c->ev_pool.push_back(a); return; }
  } else {
    b = c->ev_pool.back();
    c->ev_pool.pop_back();
  }
  cudaEventRecord(b, c->st);
  c->recs.push_back({ph, a, b});
}

// NVTX range names of the phases (profiling only: a tool such as ncu can
// then select the kernels of one phase with --nvtx-include "qrctm:x1/")
static const char* const kPhaseNames[QRCTM_NUM_PHASES] = {
    "qrctm:ct",      "qrctm:qr",     "qrctm:x1",       "qrctm:absorb",
    "qrctm:project", "qrctm:corner", "qrctm:symnorm",  "qrctm:spectrum",
    "qrctm:energy",  "qrctm:grad",   "qrctm:warmup",   "qrctm:qr_panel"};

// panel launches of the QR, timed as the nested phase QRCTM_PH_QR_PANEL
void panel_hook(void* user, int begin) {
  qrctm_ctx* c = static_cast<qrctm_ctx*>(user);
  if (begin) {
    if (c->prof) nvtxRangePushA(kPhaseNames[QRCTM_PH_QR_PANEL]);
    c->panel_ev = phase_begin(c);
  } else {
    phase_end(c, QRCTM_PH_QR_PANEL, c->panel_ev);
    c->panel_ev = nullptr;
    if (c->prof) nvtxRangePop();
  }
}

PhaseScope::PhaseScope(qrctm_ctx* c_, int ph_) : c(c_), ph(ph_), a(nullptr) {
  if (c->prof && ph >= 0 && ph < QRCTM_NUM_PHASES) nvtxRangePushA(kPhaseNames[ph]);
  a = phase_begin(c);
}

PhaseScope::~PhaseScope() {
  phase_end(c, ph, a);
  if (c->prof && ph >= 0 && ph < QRCTM_NUM_PHASES) nvtxRangePop();
}

}  // namespace qrctm

extern "C" {

const char* qrctm_version(void) { return "qrctm-b300 0.1 (sm_103a)"; }

size_t qrctm_workspace_bytes(const qrctm_config* cfg) {
  if (!cfg || !cfg_valid(*cfg)) return 0;
  return make_plan(*cfg, false, nullptr);
}

qrctm_status qrctm_create(const qrctm_config* cfg, void* workspace, size_t bytes,
                          qrctm_ctx** out) {
  if (!cfg || !out || !workspace) return QRCTM_ERR_INVALID_ARG;
  *out = nullptr;
  if (!cfg_valid(*cfg)) return QRCTM_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0) return QRCTM_ERR_INVALID_ARG;
  const size_t need = qrctm_workspace_bytes(cfg);
  if (bytes < need) return QRCTM_ERR_WORKSPACE;
  qrctm_ctx* c = new (std::nothrow) qrctm_ctx();
  if (!c) return QRCTM_ERR_INVALID_ARG;
  c->cfg = *cfg;
  if (c->cfg.check_every <= 0) c->cfg.check_every = 1;
  if (c->cfg.grad_max_iter <= 0) c->cfg.grad_max_iter = 200;
  if (c->cfg.grad_tol <= 0) c->cfg.grad_tol = 1e-12;
  c->st = reinterpret_cast<cudaStream_t>(cfg->stream);
  c->d = cfg->d; c->D = cfg->D; c->chi = cfg->chi;
  c->D2 = cfg->layers == QRCTM_LAYERS_NETWORK ? cfg->D : cfg->D * cfg->D;
  c->chi_cur = 0;
  c->split_prec = cfg->precision == QRCTM_SPLIT;
  c->ws = static_cast<char*>(workspace);
  c->ws_bytes = bytes;
  make_plan(c->cfg, true, c);
  c->iters = 0;
  c->last_delta = INFINITY;
  c->have_env = false;
  c->spec_valid = false;
  c->spec_pending = false;
  // zero the control words (error flag, QR grid barrier)
  cudaError_t e = cudaMemsetAsync(c->err, 0, 256, c->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->qrw.bar, 0, sizeof(GridBar), c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) { delete c; return QRCTM_ERR_CUDA; }
  c->qrw.err = c->err;   // QR kernels report through the context's error word
  *out = c;
  return QRCTM_OK;
}

void qrctm_destroy(qrctm_ctx* ctx) {
  if (!ctx) return;
  if (ctx->g_exec) {
    cudaStreamSynchronize(ctx->st);
    cudaGraphExecDestroy(ctx->g_exec);
  }
  if (ctx->g_stream) cudaStreamDestroy(ctx->g_stream);
  if (!ctx->recs.empty() || !ctx->ev_pool.empty()) cudaStreamSynchronize(ctx->st);
  for (auto& r : ctx->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (auto e : ctx->ev_pool) cudaEventDestroy(e);
  eigen_release(ctx);
  delete ctx;
}

qrctm_status qrctm_set_profiling(qrctm_ctx* c, int enable) {
  if (!c) return QRCTM_ERR_INVALID_ARG;
  c->prof = enable != 0;
  return QRCTM_OK;
}

qrctm_status qrctm_phase_times(qrctm_ctx* c, double* ms_out, long long* count_out) {
  if (!c) return QRCTM_ERR_INVALID_ARG;
  cudaError_t e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) return cuda_fail(c, e, "phase times");
  for (auto& r : c->recs) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess && r.ph >= 0 &&
        r.ph < QRCTM_NUM_PHASES) {
      c->ph_ms[r.ph] += ms;
      c->ph_n[r.ph] += 1;
    }
    c->ev_pool.push_back(r.a);
    c->ev_pool.push_back(r.b);
  }
  c->recs.clear();
  for (int i = 0; i < QRCTM_NUM_PHASES; ++i) {
    if (ms_out) ms_out[i] = c->ph_ms[i];
    if (count_out) count_out[i] = c->ph_n[i];
    c->ph_ms[i] = 0.0;
    c->ph_n[i] = 0;
  }
  return QRCTM_OK;
}

unsigned long long qrctm_kernel_launches(void) { return launches_so_far(); }

int qrctm_iterations(const qrctm_ctx* ctx) { return ctx ? ctx->iters : 0; }

const char* qrctm_last_error(const qrctm_ctx* ctx) {
  return ctx ? ctx->last_error.c_str() : "null context";
}

}  // extern "C"

namespace {

// ||X - sym(X)|| <= 1e-12 ||X|| for X = ld rank-5 slices (d x D^4) of the
// iPEPS tensor, or the network tensor (one slice, bond D2).
qrctm_status check_c4v(qrctm_ctx* c, const double* X, int ld) {
  const int bond = c->network ? c->D2 : c->D;
  const long long n = (long long)ld * bond * bond * bond * bond;
  cudaError_t e;
  if ((e = c4v_symmetrize(ld, bond, X, c->tmpA, c->st)) != cudaSuccess)
    return cuda_fail(c, e, "sym A");
  if ((e = axpby(c->tmpA, X, 1.0, -1.0, n, c->st)) != cudaSuccess)
    return cuda_fail(c, e, "sym A");
  if ((e = sum_squares_partials(c->tmpA, n, c->partials, 64, c->st)) != cudaSuccess)
    return cuda_fail(c, e, "sym A");
  if ((e = sum_squares_partials(X, n, c->partials + 64, 64, c->st)) != cudaSuccess)
    return cuda_fail(c, e, "sym A");
  double h[128];
  if ((e = cudaMemcpyAsync(h, c->partials, sizeof(h), cudaMemcpyDeviceToHost, c->st)) !=
      cudaSuccess)
    return cuda_fail(c, e, "sym A");
  if ((e = cudaStreamSynchronize(c->st)) != cudaSuccess) return cuda_fail(c, e, "sym A");
  double dsym = 0, nrm = 0;
  for (int i = 0; i < 64; ++i) { dsym += h[i]; nrm += h[64 + i]; }
  if (!(nrm > 0) || !std::isfinite(nrm))
    return set_err(c, QRCTM_ERR_NUMERIC, "tensor has zero or non-finite norm");
  if (std::sqrt(dsym) > 1e-12 * std::sqrt(nrm))
    return set_err(c, QRCTM_ERR_NOT_SYMMETRIC, "tensor is not C4v symmetric");
  return QRCTM_OK;
}

// (C, T) <- sym_norm of the raw boundary in (Craw, Traw) at chi = D2, then
// the warm-up steps growing chi to the target.
qrctm_status bulk_boundary_warmup(qrctm_ctx* c) {
  const int D2 = c->D2;
  cudaError_t e;
  c->chi_cur = D2;
  if ((e = sym_norm_env(c->Craw, c->Traw, c->C, c->T, D2, D2, c->partials, c->err, c->st)) !=
      cudaSuccess)
    return cuda_fail(c, e, "init env");
  int nw = c->cfg.warmup_steps;
  if (nw == 0) {
    long long cc = c->chi_cur;
    while (cc < c->chi && D2 > 1) { cc *= D2; ++nw; }
    if (nw < 2) nw = 2;
  }
  PhaseScope ps(c, QRCTM_PH_WARMUP);
  for (int w = 0; w < nw; ++w) {
    int ci = c->chi_cur;
    int co = (int)std::min<long long>(c->chi, (long long)ci * D2);
    // the standard method warms up with its own (exact) steps
    if ((e = (c->cfg.method == QRCTM_METHOD_EIGEN) ? eigen_step(c, ci, co)
                                                   : warmup_step(c, ci, co)) != cudaSuccess)
      return cuda_fail(c, e, "warm-up");
  }
  c->iters = 0;
  return QRCTM_OK;
}

}  // namespace

namespace qrctm {

// One QR-CTMRG step, replayed from a CUDA graph: the ~45 launches of a step
// (cooperative panel launches and memsets included) are captured once per
// environment bond on a stream of the context and replayed on its stream, so
// that the GPU runs them back to back without per-launch gaps.  Capture runs
// nothing; every argument of the step (workspace pointers, shapes, tensor
// maps) is fixed for a context and bond.  Eager launches when profiling (the
// phase events would be captured) or when capture is not possible.
cudaError_t qr_step_eager(qrctm_ctx* c) { return c->split_prec ? qr_step_split(c) : qr_step(c); }

cudaError_t qr_step_graph(qrctm_ctx* c) {
  if (c->prof || c->graph_off) return qr_step_eager(c);
  if (!c->g_exec || c->g_chi != c->chi_cur) {
    if (c->g_exec) {
      cudaGraphExecDestroy(c->g_exec);
      c->g_exec = nullptr;
    }
    cudaError_t e = cudaSuccess;
    if (!c->g_stream) e = cudaStreamCreateWithFlags(&c->g_stream, cudaStreamNonBlocking);
    cudaGraph_t g = nullptr;
    const int it0 = c->iters;
    const unsigned long long l0 = launches_so_far();
    if (e == cudaSuccess) e = cudaStreamBeginCapture(c->g_stream, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
      cudaStream_t saved = c->st;
      c->st = c->g_stream;
      const cudaError_t es = qr_step_eager(c);
      c->st = saved;
      e = cudaStreamEndCapture(c->g_stream, &g);
      if (es != cudaSuccess) e = es;
    }
    c->iters = it0;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c->g_exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      cudaGetLastError();
      c->g_exec = nullptr;
      c->graph_off = true;
      return qr_step_eager(c);
    }
    c->g_launches = launches_so_far() - l0;
    c->g_chi = c->chi_cur;
  }
  const cudaError_t e = cudaGraphLaunch(c->g_exec, c->st);
  if (e != cudaSuccess) return e;
  note_launch(c->g_launches);
  c->iters += 1;
  return cudaSuccess;
}

}  // namespace qrctm

namespace {

// First spectrum of the new environment; the context is ready to step.
qrctm_status finish_init(qrctm_ctx* c) {
  // The spectrum of the fresh corner is taken at the first convergence test,
  // in the same launches as the then-current corner's (one tridiagonalisation
  // latency instead of two); until then the corner waits in C_init.
  cudaError_t e;
  if ((e = cudaMemcpyAsync(c->C_init, c->C, sizeof(double) * (size_t)c->chi_cur * c->chi_cur,
                           cudaMemcpyDeviceToDevice, c->st)) != cudaSuccess)
    return cuda_fail(c, e, "init env");
  c->chi_init = c->chi_cur;
  qrctm_status s = sync_check(c, "init env");
  if (s != QRCTM_OK) return s;
  c->spec_pending = true;
  c->spec_valid = true;
  c->have_env = true;
  return QRCTM_OK;
}

}  // namespace

extern "C" {

qrctm_status qrctm_init_env(qrctm_ctx* c, const double* A, const double* C0, const double* T0) {
  if (!c || !A) return QRCTM_ERR_INVALID_ARG;
  if (c->network)
    return set_err(c, QRCTM_ERR_INVALID_ARG, "NETWORK layers: use qrctm_init_env_network");
  if ((C0 == nullptr) != (T0 == nullptr))
    return set_err(c, QRCTM_ERR_INVALID_ARG, "C0 and T0 must both be given or both NULL");
  const int d = c->d, D = c->D, D2 = c->D2;
  const long long nA = (long long)d * D2 * D2;
  c->have_env = false;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(c->A, A, sizeof(double) * nA, cudaMemcpyDeviceToDevice, c->st)) !=
      cudaSuccess)
    return cuda_fail(c, e, "copy A");
  qrctm_status s0 = check_c4v(c, c->A, d);
  if (s0 != QRCTM_OK) return s0;
  if (!c->split_layers) {
    if ((e = double_layer_kernel(d, D, c->A, c->a, c->st)) != cudaSuccess)
      return cuda_fail(c, e, "double layer");
  }
  if (c->split_prec) {
    if ((e = split_prepare_A(c)) != cudaSuccess) return cuda_fail(c, e, "split A");
  }
  c->iters = 0;
  c->spec_valid = false;
  c->spec_pending = false;
  if (C0 != nullptr) {
    c->chi_cur = c->chi;
    if ((e = sym_norm_env(C0, T0, c->C, c->T, c->chi, D2, c->partials, c->err, c->st)) !=
        cudaSuccess)
      return cuda_fail(c, e, "init env");
  } else {
    // boundary from the bulk tensor, chi0 = D^2 (<= chi, checked in cfg_valid)
    if ((e = init_env_kernel(d, D, c->A, c->Craw, c->Traw, c->st)) != cudaSuccess)
      return cuda_fail(c, e, "init env");
    qrctm_status s = bulk_boundary_warmup(c);
    if (s != QRCTM_OK) return s;
  }
  return finish_init(c);
}

qrctm_status qrctm_init_env_network(qrctm_ctx* c, const double* a, const double* v,
                                    const double* C0, const double* T0) {
  if (!c || !a) return QRCTM_ERR_INVALID_ARG;
  if (!c->network)
    return set_err(c, QRCTM_ERR_INVALID_ARG, "qrctm_init_env_network needs NETWORK layers");
  if ((C0 == nullptr) != (T0 == nullptr))
    return set_err(c, QRCTM_ERR_INVALID_ARG, "C0 and T0 must both be given or both NULL");
  const int b = c->D2;
  const long long na = (long long)b * b * b * b;
  c->have_env = false;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(c->a, a, sizeof(double) * na, cudaMemcpyDeviceToDevice, c->st)) !=
      cudaSuccess)
    return cuda_fail(c, e, "copy a");
  qrctm_status s = check_c4v(c, c->a, 1);
  if (s != QRCTM_OK) return s;
  c->iters = 0;
  c->spec_valid = false;
  c->spec_pending = false;
  if (C0 != nullptr) {
    c->chi_cur = c->chi;
    if ((e = sym_norm_env(C0, T0, c->C, c->T, c->chi, b, c->partials, c->err, c->st)) !=
        cudaSuccess)
      return cuda_fail(c, e, "init env");
    return finish_init(c);
  }
  if ((e = network_boundary(b, c->a, v, c->Craw, c->Traw, c->st)) != cudaSuccess)
    return cuda_fail(c, e, "init env");
  if ((s = bulk_boundary_warmup(c)) != QRCTM_OK) return s;
  return finish_init(c);
}

qrctm_status qrctm_network_observables(qrctm_ctx* c, const double* a_obs, double* ln_kappa_out,
                                       double* obs_out) {
  if (!c) return QRCTM_ERR_INVALID_ARG;
  if (!c->network)
    return set_err(c, QRCTM_ERR_INVALID_ARG, "network observables need NETWORK layers");
  if (!c->have_env) return set_err(c, QRCTM_ERR_STATE, "qrctm_init_env_network not called");
  cudaError_t e;
  {
    PhaseScope ps(c, QRCTM_PH_ENERGY);
    if ((e = network_traces(c, a_obs)) != cudaSuccess) return cuda_fail(c, e, "network traces");
  }
  double z[4] = {0, 0, 0, 0};
  if ((e = cudaMemcpyAsync(z, c->e_d, sizeof(z), cudaMemcpyDeviceToHost, c->st)) != cudaSuccess)
    return cuda_fail(c, e, "network traces");
  qrctm_status s = sync_check(c, "network traces");
  if (s != QRCTM_OK) return s;
  const double kappa = z[2] * z[0] / (z[1] * z[1]);
  if (!std::isfinite(kappa) || !(kappa > 0))
    return set_err(c, QRCTM_ERR_NUMERIC, "partition function per site not positive");
  if (ln_kappa_out) *ln_kappa_out = std::log(kappa);
  if (a_obs && obs_out) {
    const double o = z[3] / z[2];
    if (!std::isfinite(o)) return set_err(c, QRCTM_ERR_NUMERIC, "observable not finite");
    *obs_out = o;
  }
  return QRCTM_OK;
}

qrctm_status qrctm_step(qrctm_ctx* c, int n, double* delta_out) {
  if (!c || n < 0) return QRCTM_ERR_INVALID_ARG;
  if (!c->have_env) return set_err(c, QRCTM_ERR_STATE, "qrctm_init_env not called");
  cudaError_t e;
  for (int i = 0; i < n; ++i) {
    if (c->cfg.method == QRCTM_METHOD_EIGEN)
      e = eigen_step(c, c->chi_cur, (int)std::min<long long>(c->chi, (long long)c->chi_cur * c->D2));
    else
      e = qr_step_graph(c);
    if (e != cudaSuccess) return cuda_fail(c, e, "step");
  }
  if (delta_out) {
    if ((e = spectrum_check(c)) != cudaSuccess) return cuda_fail(c, e, "spectrum");
    double dlt;
    if ((e = cudaMemcpyAsync(&dlt, c->delta_d, sizeof(double), cudaMemcpyDeviceToHost, c->st)) !=
        cudaSuccess)
      return cuda_fail(c, e, "delta");
    qrctm_status s = sync_check(c, "step");
    if (s != QRCTM_OK) return s;
    c->last_delta = dlt;
    *delta_out = dlt;
    return QRCTM_OK;
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "step");
  return QRCTM_OK;
}

qrctm_status qrctm_run_to_convergence(qrctm_ctx* c, double tol, int max_iter, int* iters_out,
                                      double* delta_out) {
  if (!c) return QRCTM_ERR_INVALID_ARG;
  if (!c->have_env) return set_err(c, QRCTM_ERR_STATE, "qrctm_init_env not called");
  if (tol <= 0) tol = c->cfg.tol > 0 ? c->cfg.tol : 1e-10;
  if (max_iter <= 0) max_iter = c->cfg.max_iter > 0 ? c->cfg.max_iter : 500;
  const int ce = c->cfg.check_every;
  int done = 0;
  double dlt = INFINITY;
  qrctm_status s = QRCTM_OK;
  while (done < max_iter) {
    int n = std::min(ce, max_iter - done);
    s = qrctm_step(c, n, &dlt);
    if (s != QRCTM_OK) break;
    done += n;
    if (dlt < tol) break;
  }
  if (iters_out) *iters_out = done;
  if (delta_out) *delta_out = dlt;
  if (s != QRCTM_OK) return s;
  if (!(dlt < tol)) return set_err(c, QRCTM_ERR_NOT_CONVERGED, "max_iter reached");
  return QRCTM_OK;
}

qrctm_status qrctm_energy(qrctm_ctx* c, const qrctm_model* model, double* e_out) {
  if (!c || !model || !e_out) return QRCTM_ERR_INVALID_ARG;
  if (model->sublattice_rotation != 0 && model->sublattice_rotation != 1)
    return set_err(c, QRCTM_ERR_INVALID_ARG, "sublattice_rotation must be 0 or 1");
  c->nn_plain = model->sublattice_rotation == 0;
  if (!c->have_env) return set_err(c, QRCTM_ERR_STATE, "qrctm_init_env not called");
  if (c->d != 2) return set_err(c, QRCTM_ERR_INVALID_ARG, "the spin-1/2 energy needs d = 2");
  if (model->J2 != 0.0 && c->E3 == nullptr)
    return set_err(c, QRCTM_ERR_INVALID_ARG, "J2 != 0 needs with_nnn = 1");
  cudaError_t e;
  {
    PhaseScope ps(c, QRCTM_PH_ENERGY);
    e = energy_fp64(c, model->J1, model->J2);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "energy");
  qrctm_status s = sync_check(c, "energy");
  if (s != QRCTM_OK) return s;
  double h;
  if ((e = cudaMemcpy(&h, c->e_d, sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(c, e, "energy");
  *e_out = h;
  return QRCTM_OK;
}

qrctm_status qrctm_energy_grad(qrctm_ctx* c, const qrctm_model* model, int mode, int k_unroll,
                               double* grad, double* e_out) {
  if (!c || !model || !grad || !e_out) return QRCTM_ERR_INVALID_ARG;
  if (model->sublattice_rotation != 0 && model->sublattice_rotation != 1)
    return set_err(c, QRCTM_ERR_INVALID_ARG, "sublattice_rotation must be 0 or 1");
  c->nn_plain = model->sublattice_rotation == 0;
  if (!c->have_env) return set_err(c, QRCTM_ERR_STATE, "qrctm_init_env not called");
  if (c->d != 2) return set_err(c, QRCTM_ERR_INVALID_ARG, "the spin-1/2 energy needs d = 2");
  if (!c->G) return set_err(c, QRCTM_ERR_INVALID_ARG, "qrctm_energy_grad needs with_grad = 1");
  if (model->J2 != 0.0 && c->E3 == nullptr)
    return set_err(c, QRCTM_ERR_INVALID_ARG, "J2 != 0 needs with_nnn = 1");
  if (mode != QRCTM_GRAD_IMPLICIT && mode != QRCTM_GRAD_UNROLL)
    return set_err(c, QRCTM_ERR_INVALID_ARG, "unknown gradient mode");
  if (mode == QRCTM_GRAD_UNROLL && (k_unroll < 1 || k_unroll > kGradMaxUnroll))
    return set_err(c, QRCTM_ERR_INVALID_ARG, "k_unroll must be in 1..32");
  if (c->D < 2) return set_err(c, QRCTM_ERR_INVALID_ARG, "the gradient needs D >= 2");
  cudaError_t e;
  int iters = 0;
  double resid = 0.0, fp_resid = 0.0;
  {
    PhaseScope ps(c, QRCTM_PH_GRAD);
    // a split-precision context runs the contractions of the taped steps, of
    // the energy and of every reverse pass on the TF32x3 engine
    c->mm_split = c->split_prec && c->mm32 != nullptr;
    e = energy_grad_run(c, model->J1, model->J2, mode, k_unroll, grad, e_out, &iters, &resid,
                        &fp_resid);
    c->mm_split = false;
  }
  c->grad_iters = iters;
  c->grad_resid = resid;
  c->grad_fp_resid = fp_resid;
  if (e != cudaSuccess) return cuda_fail(c, e, "energy gradient");
  return sync_check(c, "energy gradient");
}

qrctm_status qrctm_optimize(qrctm_ctx* c, const qrctm_model* model,
                            const qrctm_lbfgs_options* opt, int n_steps, double* A,
                            double* energies, int* steps_out, int* evaluations_out) {
  if (!c || !model || !opt || !A || n_steps < 0) return QRCTM_ERR_INVALID_ARG;
  if (steps_out) *steps_out = 0;
  if (evaluations_out) *evaluations_out = 0;
  if (c->opt_hist <= 0)
    return set_err(c, QRCTM_ERR_INVALID_ARG, "qrctm_optimize needs opt_history > 0");
  const int hist = opt->history > 0 ? std::min(opt->history, c->opt_hist) : c->opt_hist;
  const int k = opt->k_unroll > 0 ? opt->k_unroll : 10;
  const int nograd = opt->nograd_steps;
  const int max_ls = opt->max_ls > 0 ? opt->max_ls : 10;
  const double c1 = opt->c1 > 0 ? opt->c1 : 1e-4;
  const double step0 = opt->step0 > 0 ? opt->step0 : 0.1;
  const double env_tol = opt->env_tol > 0 ? opt->env_tol : (c->cfg.tol > 0 ? c->cfg.tol : 1e-10);
  const int env_max = opt->env_max_iter > 0 ? opt->env_max_iter
                                            : (c->cfg.max_iter > 0 ? c->cfg.max_iter : 500);
  if (nograd < 0 || k > kGradMaxUnroll)
    return set_err(c, QRCTM_ERR_INVALID_ARG, "nograd_steps >= 0 and k_unroll <= 32");
  const int n = c->d * c->D2 * c->D2;
  const long long nC = (long long)c->chi * c->chi, nT = (long long)c->chi * c->D2 * c->chi;
  cudaStream_t st = c->st;
  cudaError_t e;
  int evals = 0;
  auto dcopy = [&](double* dst, const double* src, long long cnt) {
    return cudaMemcpyAsync(dst, src, sizeof(double) * cnt, cudaMemcpyDeviceToDevice, st);
  };
  // one evaluation at X: environment (reused or fresh), untracked steps,
  // energy and gradient through k tracked steps into opt_gt, the
  // environment after them into (opt_Cc, opt_Tc)
  auto evaluate = [&](const double* X, bool fresh, double* E) -> qrctm_status {
    qrctm_status s;
    if (fresh) {
      if ((s = qrctm_init_env(c, X, nullptr, nullptr)) != QRCTM_OK) return s;
      int it;
      double dl;
      s = qrctm_run_to_convergence(c, env_tol, env_max, &it, &dl);
      if (s != QRCTM_OK && s != QRCTM_ERR_NOT_CONVERGED) return s;
    } else {
      if ((s = qrctm_init_env(c, X, c->opt_Cp, c->opt_Tp)) != QRCTM_OK) return s;
    }
    if (nograd > 0 && (s = qrctm_step(c, nograd, nullptr)) != QRCTM_OK) return s;
    c->grad_keep_env = true;
    s = qrctm_energy_grad(c, model, QRCTM_GRAD_UNROLL, k, c->opt_gt, E);
    c->grad_keep_env = false;
    if (s != QRCTM_OK) return s;
    if (c->chi_cur != c->chi)
      return set_err(c, QRCTM_ERR_INVALID_ARG, "the warm-up did not reach chi");
    if ((e = dcopy(c->opt_Cc, c->C, nC)) != cudaSuccess) return cuda_fail(c, e, "optimize");
    if ((e = dcopy(c->opt_Tc, c->T, nT)) != cudaSuccess) return cuda_fail(c, e, "optimize");
    ++evals;
    if (evaluations_out) *evaluations_out = evals;
    return QRCTM_OK;
  };
  // accept the last evaluation at X (= opt_xt, or opt_x at the start)
  auto accept = [&](bool from_trial) -> cudaError_t {
    cudaError_t r = cudaSuccess;
    if (from_trial) r = dcopy(c->opt_x, c->opt_xt, n);
    if (r == cudaSuccess) r = dcopy(c->opt_g, c->opt_gt, n);
    if (r == cudaSuccess) r = dcopy(c->opt_Cp, c->opt_Cc, nC);
    if (r == cudaSuccess) r = dcopy(c->opt_Tp, c->opt_Tc, nT);
    return r;
  };
  auto read_out = [&](double* h, int cnt) -> cudaError_t {
    cudaError_t r = cudaMemcpyAsync(h, c->opt_out, sizeof(double) * cnt, cudaMemcpyDeviceToHost, st);
    return r == cudaSuccess ? cudaStreamSynchronize(st) : r;
  };
  if ((e = dcopy(c->opt_x, A, n)) != cudaSuccess) return cuda_fail(c, e, "optimize");
  double E = 0.0;
  qrctm_status s = evaluate(c->opt_x, true, &E);
  if (s != QRCTM_OK) return s;
  if ((e = accept(false)) != cudaSuccess) return cuda_fail(c, e, "optimize");
  if (energies) energies[0] = E;
  int cnt = 0, head = 0, steps = 0;
  qrctm_status result = QRCTM_OK;
  for (int it = 0; it < n_steps; ++it) {
    double o[3];
    if ((e = lbfgs_direction(n, cnt, head, hist, c->opt_S, c->opt_Y, c->opt_g, c->opt_q,
                             c->opt_p, c->opt_out, st)) != cudaSuccess ||
        (e = read_out(o, 2)) != cudaSuccess)
      return cuda_fail(c, e, "optimize direction");
    if (!(o[0] < 0.0) && cnt > 0) {
      cnt = 0;   // not a descent direction: drop the history, steepest descent
      if ((e = lbfgs_direction(n, 0, head, hist, c->opt_S, c->opt_Y, c->opt_g, c->opt_q,
                               c->opt_p, c->opt_out, st)) != cudaSuccess ||
          (e = read_out(o, 2)) != cudaSuccess)
        return cuda_fail(c, e, "optimize direction");
    }
    const double gp = o[0], pp = o[1];
    if (!(pp > 0.0)) break;   // zero gradient
    if (!std::isfinite(gp) || !std::isfinite(pp))
      return set_err(c, QRCTM_ERR_NUMERIC, "non-finite search direction");
    double alpha = cnt > 0 ? 1.0 : step0 / std::sqrt(pp);
    bool ok = false;
    double Et = 0.0;
    for (int t = 0; t < max_ls; ++t) {
      if ((e = lbfgs_trial(n, c->opt_x, alpha, c->opt_p, c->opt_xt, st)) != cudaSuccess)
        return cuda_fail(c, e, "optimize trial");
      if ((s = evaluate(c->opt_xt, t > 0, &Et)) != QRCTM_OK) return s;
      if (Et <= E + c1 * alpha * gp) { ok = true; break; }
      alpha *= 0.5;
    }
    if (!ok) {
      result = set_err(c, QRCTM_ERR_NOT_CONVERGED, "line search found no decrease");
      break;
    }
    if ((e = lbfgs_pair(n, c->opt_xt, c->opt_x, c->opt_gt, c->opt_g,
                        c->opt_S + (size_t)head * n, c->opt_Y + (size_t)head * n, c->opt_out,
                        st)) != cudaSuccess ||
        (e = read_out(o, 3)) != cudaSuccess)
      return cuda_fail(c, e, "optimize pair");
    if (o[0] > 1e-10 * std::sqrt(o[1] * o[2])) {
      head = (head + 1) % hist;
      cnt = std::min(cnt + 1, hist);
    }
    if ((e = accept(true)) != cudaSuccess) return cuda_fail(c, e, "optimize");
    E = Et;
    ++steps;
    if (energies) energies[steps] = E;
    if (steps_out) *steps_out = steps;
  }
  if ((e = dcopy(A, c->opt_x, n)) != cudaSuccess) return cuda_fail(c, e, "optimize");
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(c, e, "optimize");
  return result;
}

int qrctm_grad_iterations(const qrctm_ctx* ctx) { return ctx ? ctx->grad_iters : 0; }

double qrctm_grad_residual(const qrctm_ctx* ctx) { return ctx ? ctx->grad_resid : 0.0; }

double qrctm_grad_fixed_point_residual(const qrctm_ctx* ctx) {
  return ctx ? ctx->grad_fp_resid : 0.0;
}

qrctm_status qrctm_get_env(qrctm_ctx* c, double* C, double* T, double* spectrum_host) {
  if (!c) return QRCTM_ERR_INVALID_ARG;
  if (!c->have_env) return set_err(c, QRCTM_ERR_STATE, "qrctm_init_env not called");
  cudaError_t e;
  const long long nC = (long long)c->chi_cur * c->chi_cur;
  const long long nT = (long long)c->chi_cur * c->D2 * c->chi_cur;
  if (C && (e = cudaMemcpyAsync(C, c->C, sizeof(double) * nC, cudaMemcpyDeviceToDevice, c->st)) !=
               cudaSuccess)
    return cuda_fail(c, e, "get env");
  if (T && (e = cudaMemcpyAsync(T, c->T, sizeof(double) * nT, cudaMemcpyDeviceToDevice, c->st)) !=
               cudaSuccess)
    return cuda_fail(c, e, "get env");
  if (spectrum_host) {
    if ((e = spectrum_check(c)) != cudaSuccess) return cuda_fail(c, e, "spectrum");
    qrctm_status s = sync_check(c, "spectrum");
    if (s != QRCTM_OK) return s;
    if ((e = cudaMemcpy(spectrum_host, c->s_cur, sizeof(double) * c->chi_cur,
                        cudaMemcpyDeviceToHost)) != cudaSuccess)
      return cuda_fail(c, e, "spectrum");
  }
  return sync_check(c, "get env");
}

qrctm_status qrctm_init_env_host(qrctm_ctx* c, const double* A, const double* C0,
                                 const double* T0) {
  if (!c || !A) return QRCTM_ERR_INVALID_ARG;
  if (c->network)
    return set_err(c, QRCTM_ERR_INVALID_ARG, "NETWORK layers: use qrctm_init_env_network");
  if ((C0 == nullptr) != (T0 == nullptr))
    return set_err(c, QRCTM_ERR_INVALID_ARG, "C0 and T0 must both be given or both NULL");
  const long long nA = (long long)c->d * c->D2 * c->D2;
  const long long nC = (long long)c->chi * c->chi, nT = (long long)c->chi * c->D2 * c->chi;
  // staging: A in the X1 scratch (chi^2 D^4 >= d D^4 doubles, unused until a
  // step runs), C0 and T0 in the raw environment buffers (the inputs of the
  // symmetrise-and-normalise kernel that qrctm_init_env applies to them)
  cudaError_t e = cudaMemcpyAsync(c->X1, A, sizeof(double) * nA, cudaMemcpyHostToDevice, c->st);
  if (e == cudaSuccess && C0)
    e = cudaMemcpyAsync(c->Craw, C0, sizeof(double) * nC, cudaMemcpyHostToDevice, c->st);
  if (e == cudaSuccess && T0)
    e = cudaMemcpyAsync(c->Traw, T0, sizeof(double) * nT, cudaMemcpyHostToDevice, c->st);
  if (e != cudaSuccess) return cuda_fail(c, e, "copy host inputs");
  return qrctm_init_env(c, c->X1, C0 ? c->Craw : nullptr, T0 ? c->Traw : nullptr);
}

qrctm_status qrctm_get_env_host(qrctm_ctx* c, double* C, double* T, double* spectrum_host) {
  if (!c) return QRCTM_ERR_INVALID_ARG;
  if (!c->have_env) return set_err(c, QRCTM_ERR_STATE, "qrctm_init_env not called");
  cudaError_t e;
  const long long nC = (long long)c->chi_cur * c->chi_cur;
  const long long nT = (long long)c->chi_cur * c->D2 * c->chi_cur;
  if (C && (e = cudaMemcpyAsync(C, c->C, sizeof(double) * nC, cudaMemcpyDeviceToHost, c->st)) !=
               cudaSuccess)
    return cuda_fail(c, e, "get env");
  if (T && (e = cudaMemcpyAsync(T, c->T, sizeof(double) * nT, cudaMemcpyDeviceToHost, c->st)) !=
               cudaSuccess)
    return cuda_fail(c, e, "get env");
  // the spectrum (if asked) and the synchronisation that completes the copies
  return qrctm_get_env(c, nullptr, nullptr, spectrum_host);
}

size_t qrctm_c4v_symmetrize_workspace_bytes(void) { return 256 * sizeof(double); }

qrctm_status qrctm_c4v_symmetrize(int d, int D, const double* X, double* Y, int normalize,
                                  void* workspace, size_t bytes, void* stream) {
  if (d < 1 || D < 1 || !X || !Y || X == Y) return QRCTM_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (normalize && (!workspace || bytes < qrctm_c4v_symmetrize_workspace_bytes()))
    return QRCTM_ERR_WORKSPACE;
  cudaError_t e = c4v_symmetrize(d, D, X, Y, s);
  if (e != cudaSuccess) return QRCTM_ERR_CUDA;
  if (normalize) {
    double* parts = static_cast<double*>(workspace);
    int* err = reinterpret_cast<int*>(parts + 128);
    const long long n = (long long)d * D * D * D * D;
    if ((e = cudaMemsetAsync(err, 0, sizeof(int), s)) != cudaSuccess) return QRCTM_ERR_CUDA;
    if ((e = sum_squares_partials(Y, n, parts, 64, s)) != cudaSuccess) return QRCTM_ERR_CUDA;
    if ((e = scale_by_inv_norm(Y, Y, n, parts, 64, err, s)) != cudaSuccess) return QRCTM_ERR_CUDA;
    int flag = 0;
    if ((e = cudaMemcpyAsync(&flag, err, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
      return QRCTM_ERR_CUDA;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return QRCTM_ERR_CUDA;
    if (flag) return QRCTM_ERR_NUMERIC;
  }
  return QRCTM_OK;
}

namespace {
qrctm_status gemm_tf32x3_impl(int M, int N, int K, const float* A, const float* A_lo,
                              long long lda, const float* B, const float* B_lo, long long ldb,
                              double* C, long long ldc, float* work, long long work_elems,
                              int* err_word, void* stream) {
  if (M < 1 || N < 1 || K < 1 || !A || !B || !C || !err_word) return QRCTM_ERR_INVALID_ARG;
  if (lda < K || ldb < K || ldc < N || (lda % 4) || (ldb % 4)) return QRCTM_ERR_INVALID_ARG;
  if (A_lo && !B_lo) return QRCTM_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  TcGemm g{};
  g.A = TcOperand{A, M, K, lda, 1, 0, A_lo};
  g.B = TcOperand{B, N, K, ldb, 1, 0, B_lo};
  g.M = M; g.N = N; g.K = K; g.batch = 1;
  g.C = C; g.c_fp64 = true;
  g.c_m = im1(ldc); g.c_n = im1(1); g.c_b = im0();
  g.alpha = 1.0; g.beta = 0.0;
  g.err = err_word;
  g.part = work;
  g.part_elems = work ? work_elems : 0;
  if (cudaMemsetAsync(err_word, 0, sizeof(int), s) != cudaSuccess) return QRCTM_ERR_CUDA;
  cudaError_t e = gemm_tc(g, s);
  if (e == cudaErrorInvalidValue) return QRCTM_ERR_INVALID_ARG;
  if (e != cudaSuccess) return QRCTM_ERR_CUDA;
  int flag = 0;
  if (cudaMemcpyAsync(&flag, err_word, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return QRCTM_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return QRCTM_ERR_CUDA;
  if (flag) return (flag & ERRF_TIMEOUT) ? QRCTM_ERR_TIMEOUT : QRCTM_ERR_NUMERIC;
  return QRCTM_OK;
}
}  // namespace

qrctm_status qrctm_gemm_tf32x3(int M, int N, int K, const float* A, long long lda, const float* B,
                               long long ldb, double* C, long long ldc, float* work,
                               long long work_elems, int* err_word, void* stream) {
  return gemm_tf32x3_impl(M, N, K, A, nullptr, lda, B, nullptr, ldb, C, ldc, work, work_elems,
                          err_word, stream);
}

qrctm_status qrctm_gemm_tf32x3_presplit(int M, int N, int K, const float* A, const float* A_lo,
                                        long long lda, const float* B, const float* B_lo,
                                        long long ldb, double* C, long long ldc, float* work,
                                        long long work_elems, int* err_word, void* stream) {
  if (!B_lo) return QRCTM_ERR_INVALID_ARG;
  return gemm_tf32x3_impl(M, N, K, A, A_lo, lda, B, B_lo, ldb, C, ldc, work, work_elems,
                          err_word, stream);
}

qrctm_status qrctm_tf32_split(long long rows, int cols, float* x, long long ld, float* lo,
                              void* stream) {
  if (rows < 0 || cols < 0 || !x || !lo || ld < cols) return QRCTM_ERR_INVALID_ARG;
  if (rows * (long long)cols >= (1ll << 32)) return QRCTM_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (split_f32(x, lo, rows, cols, ld, s) != cudaSuccess) return QRCTM_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return QRCTM_ERR_CUDA;
  return QRCTM_OK;
}

size_t qrctm_qr_workspace_bytes(int m, int n) {
  if (m < n || n < 1 || n > 2048) return 0;
  return qr_work_bytes(m, n);
}

qrctm_status qrctm_householder_qr(int m, int n, const double* M, double* Q, double* R,
                                  void* workspace, size_t bytes, void* stream) {
  return qrctm_householder_qr_bounded(m, n, M, Q, R, workspace, bytes, stream, 0, 0);
}

qrctm_status qrctm_householder_qr_bounded(int m, int n, const double* M, double* Q, double* R,
                                          void* workspace, size_t bytes, void* stream,
                                          long long wait_spins, int extra_arrivals) {
  if (m < n || n < 1 || n > 2048 || !M || !Q || !R || !workspace) return QRCTM_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0) return QRCTM_ERR_INVALID_ARG;
  if (wait_spins < 0 || extra_arrivals < 0 || extra_arrivals > 1024) return QRCTM_ERR_INVALID_ARG;
  if (bytes < qrctm_qr_workspace_bytes(m, n)) return QRCTM_ERR_WORKSPACE;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  QrWork w = qr_carve(workspace, m, n);
  if (wait_spins > 0) w.wait_spins = wait_spins;
  w.wait_extra = (unsigned)extra_arrivals;
  cudaError_t e = householder_qr_f64(m, n, M, Q, R, w, s);
  if (e != cudaSuccess) return QRCTM_ERR_CUDA;
  int flag = 0;
  if ((e = cudaMemcpyAsync(&flag, w.err, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return QRCTM_ERR_CUDA;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return QRCTM_ERR_CUDA;
  if (flag) {
    cudaMemsetAsync(w.err, 0, sizeof(int), s);
    if (flag & ERRF_TIMEOUT) cudaMemsetAsync(w.bar, 0, sizeof(GridBar), s);
    cudaStreamSynchronize(s);
    return (flag & ERRF_TIMEOUT) ? QRCTM_ERR_TIMEOUT : QRCTM_ERR_NUMERIC;
  }
  return QRCTM_OK;
}

}  // extern "C"
