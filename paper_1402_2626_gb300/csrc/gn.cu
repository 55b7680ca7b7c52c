// gn.cu — host side of the C ABI declared in include/gn.h: loading a system in
// sparse distributed form (Section 1, Problem Statement), per-precision
// workspaces, and the Newton driver (Section 4) that keeps every step on the
// device as one CUDA graph replayed per step.
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "internal.h"

namespace gn {

template <typename T>
static gn_status dalloc(T **p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  if (cudaMalloc((void **)p, sizeof(T) * count) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return GN_ENOMEM;
  }
  return GN_OK;
}

template <typename T>
static gn_status upload(T **p, const T *h, size_t count) {
  gn_status e = dalloc(p, count);
  if (e) return e;
  if (count && cudaMemcpy(*p, h, sizeof(T) * count, cudaMemcpyHostToDevice) != cudaSuccess)
    return GN_ECUDA;
  return GN_OK;
}

static void ws_free(Workspace &w) {
  if (w.step_exec) cudaGraphExecDestroy(w.step_exec);
  if (w.cq_exec) cudaGraphExecDestroy(w.cq_exec);
  if (w.ref_exec) cudaGraphExecDestroy(w.ref_exec);
  cudaFree(w.pow);
  cudaFree(w.stage_val);
  cudaFree(w.stage_d);
  cudaFree(w.Ab);
  cudaFree(w.R);
  cudaFree(w.dx);
  cudaFree(w.lam);
  cudaFree(w.xmix);
  cudaFree(w.rinv);
  cudaFree(w.norms);
  cudaFree(w.status);
  cudaFree(w.flags);
  cudaFree(w.Rm);
  cudaFree(w.Zs);
  cudaFree(w.Xinv);
  cudaFree(w.cq_scratch);
  if (w.cq_ev[0]) cudaEventDestroy(w.cq_ev[0]);
  if (w.cq_ev[1]) cudaEventDestroy(w.cq_ev[1]);
  if (w.cq_side) cudaStreamDestroy(w.cq_side);
  if (w.h_norms) cudaFreeHost(w.h_norms);
  if (w.h_status) cudaFreeHost(w.h_status);
  w = Workspace();
}

gn_status workspace_get(gn_system *s, int L, Workspace **out) {
  Workspace &w = s->ws[L];
  *out = &w;
  if (w.ready) return GN_OK;
  const size_t W = 2 * (size_t)L;
  const size_t n = s->n, N = s->N;
  gn_status e = GN_OK;
  const size_t SW = stage_words(L);
  if (!e) e = dalloc(&w.pow, SW * n * s->pmax);
  if (!e) e = dalloc(&w.stage_val, SW * s->T);
  if (!e) e = dalloc(&w.stage_d, SW * s->nnz);
  if (!e) e = dalloc(&w.Ab, W * N * (n + 1));
  if (!e) e = dalloc(&w.R, W * (n + 1) * (n + 1));
  if (!e) e = dalloc(&w.dx, W * n);
  if (!e) e = dalloc(&w.lam, W * N);
  if (!e) e = dalloc(&w.xmix, 2 * n);
  if (!e) e = dalloc(&w.rinv, lstsq_scratch_doubles(s->n, L));
  if (!e) e = dalloc(&w.norms, 3 * GN_REPORT_MAX);
  if (!e) e = dalloc(&w.status, 2);
  if (!e) e = dalloc(&w.flags, (n + 1) * MGS_FLAGS_PER_COLUMN);
  if (!e) e = dalloc(&w.Rm, W * (n + 1) * (n + 1));
  if (!e) e = dalloc(&w.Zs, (n + 1) * (L + 1));
  if (!e) e = dalloc(&w.Xinv, bs_inv_doubles(s->n, L));
  if (!e && cudaMallocHost((void **)&w.h_norms, sizeof(double) * 3 * GN_REPORT_MAX) != cudaSuccess)
    e = GN_ENOMEM;
  if (!e && cudaMallocHost((void **)&w.h_status, sizeof(int32_t) * 2) != cudaSuccess) e = GN_ENOMEM;
  if (!e && cudaMemset(w.status, 0, sizeof(int32_t) * 2) != cudaSuccess) e = GN_ECUDA;
  if (e) {
    cudaGetLastError();
    ws_free(w);
    return e;
  }
  // query cluster occupancy now: never during a stream capture
  mgs_flow_clusters(L);
  backsub_prepare(L);
  w.ready = true;
  return GN_OK;
}

}  // namespace gn

using namespace gn;

static bool valid_prec(int p) { return p == 1 || p == 2 || p == 4; }

extern "C" {

const char *gn_status_str(gn_status st) {
  switch (st) {
    case GN_OK: return "ok";
    case GN_EINVAL: return "invalid argument";
    case GN_ENOMEM: return "out of memory";
    case GN_ECUDA: return "CUDA error";
    case GN_ESINGULAR: return "singular Jacobian";
    case GN_ENOCONV: return "no convergence";
    case GN_ENONFINITE: return "non-finite value";
    case GN_ETIMEOUT: return "device wait timed out";
  }
  return "unknown status";
}

int32_t gn_version(void) { return 100; }

gn_status gn_system_create(gn_system **out, int32_t N, int32_t n, int64_t T,
                           const int64_t *h_poly_ptr, const int64_t *h_mono_ptr,
                           const int32_t *h_var, const uint8_t *h_exp, const double *h_coef,
                           int32_t coef_limbs) {
  gn::Range nvtx_range("gn_system_create");
  if (!out) return GN_EINVAL;
  *out = nullptr;
  if (n < 1 || N < n || T < 0 || n >= (1 << 24)) return GN_EINVAL;
  if (!h_poly_ptr || !h_mono_ptr || (T > 0 && !h_coef) || !valid_prec(coef_limbs)) return GN_EINVAL;
  if (h_poly_ptr[0] != 0 || h_poly_ptr[N] != T || h_mono_ptr[0] != 0) return GN_EINVAL;
  for (int32_t i = 0; i < N; i++)
    if (h_poly_ptr[i + 1] < h_poly_ptr[i]) return GN_EINVAL;
  for (int64_t t = 0; t < T; t++)
    if (h_mono_ptr[t + 1] < h_mono_ptr[t]) return GN_EINVAL;
  const int64_t nnz = h_mono_ptr[T];
  if (nnz >= ((int64_t)1 << 31) || T >= ((int64_t)1 << 31)) return GN_EINVAL;
  if (nnz > 0 && (!h_var || !h_exp)) return GN_EINVAL;

  // validate supports: variables in range, distinct within a monomial, exponents >= 1
  std::vector<int64_t> seen(n, -1);
  int32_t kmax = 0, dmax = 1;
  for (int64_t t = 0; t < T; t++) {
    int32_t k = (int32_t)(h_mono_ptr[t + 1] - h_mono_ptr[t]);
    kmax = std::max(kmax, k);
    for (int64_t o = h_mono_ptr[t]; o < h_mono_ptr[t + 1]; o++) {
      int32_t v = h_var[o];
      if (v < 0 || v >= n || h_exp[o] < 1 || seen[v] == t) return GN_EINVAL;
      seen[v] = t;
      dmax = std::max(dmax, (int32_t)h_exp[o]);
    }
  }

  gn_system *s = new (std::nothrow) gn_system();
  if (!s) return GN_ENOMEM;
  s->N = N;
  s->n = n;
  s->T = T;
  s->nnz = nnz;
  s->kmax = kmax;
  s->dmax = dmax;
  s->pmax = std::max(dmax - 1, 1);

  std::vector<int32_t> poly_ptr(N + 1), mono_off(T + 1);
  for (int32_t i = 0; i <= N; i++) poly_ptr[i] = (int32_t)h_poly_ptr[i];
  for (int64_t t = 0; t <= T; t++) mono_off[t] = (int32_t)h_mono_ptr[t];
  std::vector<uint32_t> occ(nnz);
  for (int64_t o = 0; o < nnz; o++) occ[o] = ((uint32_t)h_var[o] << 8) | (uint32_t)h_exp[o];
  // limb-planar coefficients [limb][part][T], limbs beyond coef_limbs are 0
  std::vector<double> coef((size_t)8 * T, 0.0);
  for (int64_t t = 0; t < T; t++)
    for (int part = 0; part < 2; part++)
      for (int l = 0; l < coef_limbs; l++)
        coef[(size_t)(2 * l + part) * T + t] = h_coef[(t * 2 + part) * coef_limbs + l];

  // Jacobian pattern: occurrences bucketed by column (stable), so within a
  // column rows come in term order; runs of equal (column, row) are entries.
  std::vector<int32_t> occ_row(nnz);
  for (int32_t i = 0; i < N; i++)
    for (int64_t t = h_poly_ptr[i]; t < h_poly_ptr[i + 1]; t++)
      for (int64_t o = h_mono_ptr[t]; o < h_mono_ptr[t + 1]; o++) occ_row[o] = i;
  std::vector<int64_t> col_start(n + 1, 0);
  for (int64_t o = 0; o < nnz; o++) col_start[h_var[o] + 1]++;
  for (int32_t v = 0; v < n; v++) col_start[v + 1] += col_start[v];
  std::vector<int32_t> by_col(nnz);
  {
    std::vector<int64_t> fill(col_start.begin(), col_start.end() - 1);
    for (int64_t o = 0; o < nnz; o++) by_col[fill[h_var[o]]++] = (int32_t)o;
  }
  std::vector<int32_t> jz_row, jz_col, jz_ptr;
  for (int32_t v = 0; v < n; v++) {
    for (int64_t p = col_start[v]; p < col_start[v + 1]; p++) {
      int32_t r = occ_row[by_col[p]];
      if (p == col_start[v] || occ_row[by_col[p - 1]] != r) {
        jz_ptr.push_back((int32_t)p);
        jz_row.push_back(r);
        jz_col.push_back(v);
      }
    }
  }
  jz_ptr.push_back((int32_t)nnz);
  s->nz = (int64_t)jz_row.size();

  gn_status e = GN_OK;
  if (!e) e = upload(&s->d_poly_ptr, poly_ptr.data(), poly_ptr.size());
  if (!e) e = upload(&s->d_mono_off, mono_off.data(), mono_off.size());
  if (!e) e = upload(&s->d_occ, occ.data(), occ.size());
  if (!e) e = upload(&s->d_coef, coef.data(), coef.size());
  {
    std::vector<int32_t> lt;
    for (int64_t t = 0; t < T; t++)
      if (h_mono_ptr[t + 1] - h_mono_ptr[t] > 64) lt.push_back((int32_t)t);
    s->nlong = (int64_t)lt.size();
    if (!e && !lt.empty()) e = upload(&s->d_long, lt.data(), lt.size());
  }
  if (!e) e = upload(&s->d_jz_row, jz_row.data(), jz_row.size());
  if (!e) e = upload(&s->d_jz_col, jz_col.data(), jz_col.size());
  if (!e) e = upload(&s->d_jz_ptr, jz_ptr.data(), jz_ptr.size());
  if (!e) e = upload(&s->d_jz_occ, by_col.data(), by_col.size());
  if (e) {
    gn_system_destroy(s);
    return e;
  }
  *out = s;
  return GN_OK;
}

gn_status gn_system_destroy(gn_system *s) {
  if (!s) return GN_EINVAL;
  cudaDeviceSynchronize();
  for (int L = 0; L < 5; L++) ws_free(s->ws[L]);
  cudaFree(s->d_poly_ptr);
  cudaFree(s->d_mono_off);
  cudaFree(s->d_occ);
  cudaFree(s->d_coef);
  cudaFree(s->d_long);
  cudaFree(s->d_jz_row);
  cudaFree(s->d_jz_col);
  cudaFree(s->d_jz_ptr);
  cudaFree(s->d_jz_occ);
  delete s;
  return GN_OK;
}

gn_status gn_system_info(const gn_system *s, int32_t *N, int32_t *n, int64_t *T, int64_t *nnz,
                         int32_t *max_support) {
  if (!s) return GN_EINVAL;
  if (N) *N = s->N;
  if (n) *n = s->n;
  if (T) *T = s->T;
  if (nnz) *nnz = s->nnz;
  if (max_support) *max_support = s->kmax;
  return GN_OK;
}

gn_status gn_eval(gn_system *s, gn_prec prec, const double *d_x, double *d_f, double *d_J,
                  int64_t ldJ, void *cuda_stream) {
  gn::Range nvtx_range("gn_eval");
  if (!s || !valid_prec(prec) || !d_x || (d_J && ldJ < s->N)) return GN_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  Workspace *ws;
  gn_status e = workspace_get(s, prec, &ws);
  if (e) return e;
  if (cudaMemsetAsync(ws->status, 0, sizeof(int32_t) * 2, st) != cudaSuccess) return GN_ECUDA;
  return launch_eval_sel(s, prec, d_x, d_f, 0, d_J, ldJ, st);
}

gn_status gn_system_set_arith(gn_system *s, gn_arith arith) {
  if (!s || (arith != GN_ARITH_AUTO && arith != GN_ARITH_INT && arith != GN_ARITH_FP64))
    return GN_EINVAL;
  if (s->arith == (int32_t)arith) return GN_OK;
  s->arith = arith;
  for (Workspace &w : s->ws) w.fact = 0;
  for (Workspace &w : s->ws) {
    if (w.step_exec) {
      cudaGraphExecDestroy(w.step_exec);
      w.step_exec = nullptr;
      w.graph_x = nullptr;
    }
    if (w.cq_exec) {
      cudaGraphExecDestroy(w.cq_exec);
      w.cq_exec = nullptr;
    }
    if (w.ref_exec) {
      cudaGraphExecDestroy(w.ref_exec);
      w.ref_exec = nullptr;
      w.ref_x = nullptr;
    }
  }
  return GN_OK;
}

gn_status gn_lstsq(gn_system *s, gn_prec prec, int32_t m, int32_t n, double *d_Ab, int64_t ldAb,
                   double *d_R, double *d_dx, void *cuda_stream) {
  gn::Range nvtx_range("gn_lstsq");
  if (!s || !valid_prec(prec) || n < 1 || m < n || ldAb < m || !d_Ab || !d_R || !d_dx)
    return GN_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  Workspace *ws;
  gn_status e = workspace_get(s, prec, &ws);
  if (e) return e;
  double *scratch = ws->rinv;
  uint32_t *flags = ws->flags;
  double *Rm = ws->Rm, *Zs = ws->Zs;
  bool own = false;
  if (n > s->n) {  // larger than the system's own workspace: temporary scratch
    if (cudaMalloc((void **)&scratch, sizeof(double) * lstsq_scratch_doubles(n, prec)) != cudaSuccess) {
      cudaGetLastError();
      return GN_ENOMEM;
    }
    if (cudaMalloc((void **)&flags, sizeof(uint32_t) * (n + 1) * MGS_FLAGS_PER_COLUMN) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(scratch);
      return GN_ENOMEM;
    }
    if (cudaMalloc((void **)&Rm, sizeof(double) * 2 * prec * (size_t)(n + 1) * (n + 1)) != cudaSuccess ||
        cudaMalloc((void **)&Zs, sizeof(double) * (size_t)(n + 1) * (prec + 1)) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(scratch);
      cudaFree(flags);
      cudaFree(Rm);
      return GN_ENOMEM;
    }
    own = true;
  }
  ws->fact = 0;
  if (cudaMemsetAsync(ws->status, 0, sizeof(int32_t) * 2, st) != cudaSuccess) return GN_ECUDA;
  e = launch_lstsq(s, prec, m, n, d_Ab, ldAb, d_R, scratch, flags, Rm, Zs, own ? nullptr : ws->Xinv,
                   d_dx, ws->status, st, true);
  if (!e && cudaMemcpyAsync(ws->h_status, ws->status, sizeof(int32_t) * 2, cudaMemcpyDeviceToHost,
                            st) != cudaSuccess)
    e = GN_ECUDA;
  if (!e && cudaStreamSynchronize(st) != cudaSuccess) e = GN_ECUDA;
  if (own) {
    cudaFree(scratch);
    cudaFree(flags);
    cudaFree(Rm);
    cudaFree(Zs);
  }
  if (e) return e;
  return (gn_status)ws->h_status[0];
}

gn_status gn_mgs(gn_system *s, gn_prec prec, int32_t m, int32_t n, double *d_Ab, int64_t ldAb,
                 double *d_R, int32_t *d_status, void *cuda_stream) {
  gn::Range nvtx_range("gn_mgs");
  if (!s || !valid_prec(prec) || n < 1 || n > s->n || m < n || ldAb < m || !d_Ab || !d_R ||
      !d_status)
    return GN_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  Workspace *ws;
  gn_status e = workspace_get(s, prec, &ws);
  if (e) return e;
  ws->fact = 0;
  if (cudaMemsetAsync(ws->status, 0, sizeof(int32_t) * 2, st) != cudaSuccess) return GN_ECUDA;
  e = launch_lstsq(s, prec, m, n, d_Ab, ldAb, d_R, ws->rinv, ws->flags, ws->Rm, ws->Zs, nullptr,
                   nullptr, ws->status, st, true);
  if (e) return e;
  if (cudaMemcpyAsync(d_status, ws->status, sizeof(int32_t), cudaMemcpyDeviceToDevice, st) !=
      cudaSuccess)
    return GN_ECUDA;
  return GN_OK;
}

}  // extern "C"

namespace gn {

// One Gauss-Newton step on stream st: [J, -f] into Ab, MGS + back
// substitution into dx, x += dx.
static gn_status newton_step(gn_system *s, int L, Workspace *ws, double *d_x, cudaStream_t st) {
  const int64_t W = 2 * L;
  const int32_t N = s->N, n = s->n;
  gn_status e = launch_eval_sel(s, L, d_x, ws->Ab + (int64_t)n * N * W, 1, ws->Ab, N, st);
  if (e) return e;
  e = launch_lstsq(s, L, N, n, ws->Ab, N, ws->R, ws->rinv, ws->flags, ws->Rm, ws->Zs, ws->Xinv, ws->dx,
                   ws->status, st, false);
  if (e) return e;
  const double *fnorm = ws->rinv + (int64_t)(n + 1) * L + n;  // original norm of the b column
  return launch_update(L, n, d_x, ws->dx, fnorm, ws->norms, ws->status, st);
}

static gn_status build_graph(gn_system *s, int L, Workspace *ws, double *d_x) {
  gn::Range nvtx_range("gn_newton: capture step graph");
  if (ws->step_exec) {
    cudaGraphExecDestroy(ws->step_exec);
    ws->step_exec = nullptr;
  }
  cudaStream_t cap;
  if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return GN_ECUDA;
  gn_status e = GN_OK;
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) e = GN_ECUDA;
  if (!e) {
    e = newton_step(s, L, ws, d_x, cap);
    if (cudaStreamEndCapture(cap, &g) != cudaSuccess && !e) e = GN_ECUDA;
  }
  if (!e && cudaGraphInstantiate(&ws->step_exec, g, 0) != cudaSuccess) e = GN_ECUDA;
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cap);
  if (e) {
    cudaGetLastError();
    ws->step_exec = nullptr;
    return e;
  }
  ws->graph_x = d_x;
  return GN_OK;
}

}  // namespace gn

extern "C" gn_status gn_newton(gn_system *s, gn_prec prec, double *d_x, int32_t steps, double tol,
                               gn_report *report, void *cuda_stream) {
  gn::Range nvtx_range("gn_newton");
  if (!s || !valid_prec(prec) || !d_x || steps < 1 || steps > GN_REPORT_MAX || !(tol >= 0.0))
    return GN_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  Workspace *ws;
  gn_status e = workspace_get(s, prec, &ws);
  if (e) return e;
  if (!ws->step_exec || ws->graph_x != d_x) {
    e = build_graph(s, prec, ws, d_x);
    if (e) return e;
  }
  ws->fact = 0;
  if (cudaMemsetAsync(ws->status, 0, sizeof(int32_t) * 2, st) != cudaSuccess) return GN_ECUDA;
  if (cudaMemsetAsync(ws->norms, 0, sizeof(double) * 3 * GN_REPORT_MAX, st) != cudaSuccess)
    return GN_ECUDA;
  int32_t done = 0;
  gn_status run = GN_OK;
  bool converged = false;
  for (int32_t k = 0; k < steps; k++) {
    if (cudaGraphLaunch(ws->step_exec, st) != cudaSuccess) return GN_ECUDA;
    if (tol > 0.0) {
      if (cudaMemcpyAsync(ws->h_status, ws->status, sizeof(int32_t) * 2, cudaMemcpyDeviceToHost, st) !=
              cudaSuccess ||
          cudaMemcpyAsync(ws->h_norms, ws->norms, sizeof(double) * 3 * GN_REPORT_MAX,
                          cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        return GN_ECUDA;
      if (ws->h_status[0] != GN_OK) break;
      double dxn = ws->h_norms[3 * k + 1], xn = ws->h_norms[3 * k + 2];
      if (dxn <= tol * xn) {
        converged = true;
        break;
      }
    }
  }
  if (cudaMemcpyAsync(ws->h_status, ws->status, sizeof(int32_t) * 2, cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(ws->h_norms, ws->norms, sizeof(double) * 3 * GN_REPORT_MAX,
                      cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return GN_ECUDA;
  run = (gn_status)ws->h_status[0];
  done = ws->h_status[1];
  // the workspace now holds the factorisation of the last step's J
  if (run == GN_OK && done >= 1) {
    ws->fact_int = lstsq_int_path(s, prec, s->N, s->n) ? 1 : 0;
    ws->fact = ws->fact_int ? 1 : 2;
  }
  if (run == GN_OK && tol > 0.0 && !converged) run = GN_ENOCONV;
  if (report) {
    memset(report, 0, sizeof(*report));
    report->steps_done = done;
    report->status = run;
    for (int32_t k = 0; k < done && k < GN_REPORT_MAX; k++) {
      report->res_norm[k] = ws->h_norms[3 * k];
      report->dx_norm[k] = ws->h_norms[3 * k + 1];
    }
  }
  return run;
}
