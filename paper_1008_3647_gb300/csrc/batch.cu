// Batched two-step BiCGStab for many independent problems of uneven lattice size.
//
// All problems' vectors live in packed arenas (problem p at element offset off_p).  Every phase
// of the iteration is one launch for the whole batch per lattice-extent group (slice kernels and
// the M0^{-1} recurrence are specialised by N_x) or one launch for the whole batch (vector and
// scalar kernels), driven by device tile tables: a slice tile is (problem, first time slice), a
// vector tile (problem, start, length), a recurrence tile (problem, 32-mode block).  Per-problem
// scalars and `done` flags let converged problems drop out while the rest continue; the
// iteration body is captured once in a CUDA graph and replayed between host checks.  Tiles are
// ordered largest problem first so that the tail of every launch is made of small problems.
#include <algorithm>
#include <functional>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "blas.cuh"
#include "ufg_internal.h"
#include "launch.cuh"

using namespace ufg;

namespace {

constexpr int VT_LEN = 8192;  // elements per vector tile

enum BSlot { B_SLICE1 = 0, B_SLICE2, B_VEC1, B_VEC2, B_DOT, B_RES, B_NSLOT };
enum BOp { BOP_M = 0, BOP_MDAG = 1 };

struct Group {
  ufg_lattice* lat = nullptr;           // owns the line tables and b(k) of this (N_x, tau)
  std::vector<int> probs;
  BatchTile* tiles = nullptr;           // device slice tiles
  int ntiles = 0;
  int cta_base = 0;                     // first slice-CTA index of the group (partials)
  int2* rtiles = nullptr;               // device recurrence tiles
  int nrtiles = 0;
  int max_ntau = 0;
  int spc = 1;                          // time slices per slice tile (tune_tiles)
};

struct Arena {  // one precision's vectors, packed over all problems
  void *r = nullptr, *rhat = nullptr, *p = nullptr, *v = nullptr, *s = nullptr, *t = nullptr,
       *y = nullptr, *z = nullptr, *spec = nullptr, *wr = nullptr, *acc = nullptr, *x = nullptr,
       *rhs = nullptr;
};

struct Batch {
  int n = 0;
  std::vector<ufg_problem> pr;
  std::vector<long long> off;
  long long S = 0;
  std::vector<Group> groups;
  std::vector<int> group_of;
  BatchProb* probs = nullptr;     // device
  std::vector<BatchProb> probs_h;
  int4* vtiles = nullptr;
  int nvtiles = 0;
  int nslice_ctas = 0;
  DevScalars* scs = nullptr;
  DevScalars* scs_h = nullptr;    // pinned
  unsigned* counters = nullptr;   // per-problem CTA counters of fused scalar updates
  int* done_dummy = nullptr;
  double* w64 = nullptr;
  double* s64 = nullptr;
  float* w32 = nullptr;
  float* s32 = nullptr;
  double* c64 = nullptr;
  float* c32 = nullptr;
  Arena ar[2];
  double *x64 = nullptr, *b64 = nullptr, *r64 = nullptr, *y64 = nullptr;
  // Momentum basis (Sec. 3): while `mom` is set, every arena vector holds F x per slice, the
  // operator is the fused momentum-space M and the WCE preconditioner needs no transforms.
  bool mom = false;
  double *xm64 = nullptr, *bm64 = nullptr;  // the right-hand side and solution in that basis
  double *rc64 = nullptr, *cr64 = nullptr;  // correction round: residual copy and correction
  double* d64 = nullptr;  // mixed solves: the FP64 increment of an incremental reliable update
  double* scale = nullptr;        // per-problem scale factors (mixed precision glue), 2 n
  double* scale_h = nullptr;      // pinned
  double* parts = nullptr;
  size_t part_stride = 0;
  cudaStream_t st = nullptr;
  int pc_kind = UFG_PC_NONE;
  ufg_pc_params pc = {};
  std::map<std::string, cudaGraphExec_t> graphs;
  std::map<std::string, long long> graph_kernels;
  std::vector<void*> allocs;
  ~Batch() {
    for (auto& kv : graphs) {
      profile_graph_destroyed(kv.second);
      cudaGraphExecDestroy(kv.second);
    }
    for (void* p : allocs) cudaFree(p);
    if (scs_h) cudaFreeHost(scs_h);
    if (scale_h) cudaFreeHost(scale_h);
    for (auto& g : groups) ufg_lattice_destroy(g.lat);
    if (st) cudaStreamDestroy(st);
  }
  template <typename T>
  ufg_status alloc(T** p, size_t n_) {
    UFG_TRY(dev_alloc(p, n_));
    allocs.push_back((void*)*p);
    return UFG_OK;
  }
  double* slot(int k) { return parts + (size_t)k * part_stride; }
};

const void* fldb(Batch& B, char w, int prec) {
  switch (w) {
    case 'w': return prec ? (const void*)B.w32 : (const void*)B.w64;
    case 's': return prec ? (const void*)B.s32 : (const void*)B.s64;
  }
  return nullptr;
}

// The work of a batched launch for the kernel timer: per_site bytes for every site of the
// problems in `idx` (all problems when null) that run under exec_if, per_problem bytes each.
LaunchWork batch_work(Batch& B, const std::vector<int>* idx, int exec_if, double per_site,
                      double per_problem = 0.0) {
  LaunchWork w;
  if (!profiling()) return w;
  w.flag_dev = &B.scs[0].done;
  w.stride = sizeof(DevScalars);
  w.exec_if = exec_if;
  w.site_bytes.assign(B.n, 0.0);
  for (int i = 0; i < B.n; ++i) {
    if (idx && std::find(idx->begin(), idx->end(), i) == idx->end()) continue;
    w.site_bytes[i] = per_site * (double)B.probs_h[i].V * B.probs_h[i].ntau + per_problem;
  }
  return w;
}

ufg_status slice(Batch& B, Group& g, SliceCall c, int exec_if) {
  c.tiles = g.tiles;
  c.ntiles = g.ntiles;
  c.probs = B.probs;
  c.exec_if = exec_if;
  c.nelem = B.S;
  if (c.partials) c.partials += 2 * (size_t)g.cta_base;
  c.scs = B.scs;  // the fused scalar step and the fused direction update read them
  if (c.fop >= 0) {
    c.counters = B.counters;
    c.part_base = g.cta_base;
  }
  note_launches(1);
  KTimer kt(slice_kernel_name(c, g.lat->nx), B.st,
            batch_work(B, &g.probs, exec_if, slice_bytes_per_site(c),
                       slice_bytes_per_problem(c, g.lat->nx)));
  cudaError_t e = slice_dispatch(g.lat->nx, c, B.st);
  if (e != cudaSuccess) return cuda_fail(e, "batched slice kernel");
  return UFG_OK;
}

// out = a * (A in) + bU * U with partials (out.dotP, out.out), all groups; fop >= 0 applies that
// scalar op to each problem from the partials in the same launch
// emulate64 (FP64, momentum basis): double-float arithmetic on the FP32 pipe (slice_df.cuh)
ufg_status apply_b(Batch& B, int prec, int op, const void* in, void* out, double a, const void* U,
                   double bU, const void* dotP, bool self, double* part, int exec_if,
                   int fop = -1, bool emulate64 = false) {
  if (B.mom) {  // the fused momentum-space operator, one kernel per group
    for (auto& g : B.groups) {
      SliceCall c = base_call(g.lat, FAM_INV, prec);
      c.fam = FAM_M1W;
      c.emulate64 = (emulate64 && prec == 0) ? 1 : 0;
      c.coef2 = base_call(g.lat, FAM_FWD, prec).coef;
      c.m1w_full = 1;
      c.in = in;
      c.pre = fldb(B, 'w', prec);
      const void* bk = prec ? (const void*)g.lat->bk32 : (const void*)g.lat->bk64;
      if (op == BOP_M) c.bkpost = bk;
      else c.bkpre = bk;
      c.shift = op == BOP_M ? -1 : +1;
      c.a = 1.0;
      c.full_scale = a;
      c.out = out;
      c.U = U;
      c.bU = bU;
      c.dotP = dotP;
      c.want_dotP = dotP != nullptr;
      c.want_self = self;
      c.partials = part;
      c.fop = fop;
      UFG_TRY(slice(B, g, c, exec_if));
    }
    return UFG_OK;
  }
  for (auto& g : B.groups) {
    SliceCall c = base_call(g.lat, FAM_KIN, prec);
    c.in = in;
    c.id = in;
    if (op == BOP_M) {
      c.pre = fldb(B, 'w', prec);
      c.shift = -1;
    } else {
      c.post = fldb(B, 'w', prec);
      c.shift = +1;
    }
    c.out = out;
    c.a = a;
    c.U = U;
    c.bU = bU;
    c.dotP = dotP;
    c.want_dotP = dotP != nullptr;
    c.want_self = self;
    c.partials = part;
    c.fop = fop;
    UFG_TRY(slice(B, g, c, exec_if));
  }
  return UFG_OK;
}

ufg_status vecb(Batch& B, int prec, int op, int exec_if, const void* a, const void* b,
                const void* c, const void* d, const void* e, const void* f, double* part,
                int fop = -1) {
  note_launches(1);
  KTimer kt(vec_op_name(op, prec), B.st,
            batch_work(B, nullptr, exec_if,
                       (prec ? 4.0 : 8.0) * vec_op_arrays(op, a != nullptr, c != nullptr)));
  cudaError_t err = launch_vec_batch(prec, op, B.vtiles, B.nvtiles, B.scs, exec_if, (void*)a,
                                     (void*)b, (void*)c, (void*)d, (void*)e, (void*)f, part, B.st,
                                     fop, B.probs, B.counters);
  if (err != cudaSuccess) return cuda_fail(err, "batched vector kernel");
  return UFG_OK;
}

ufg_status scalb(Batch& B, int op, const double* part, int kind, const double* part2, int kind2,
                 int exec_if) {
  note_launches(1);
  KTimer kt("scalar", B.st, LaunchWork{});
  cudaError_t err = launch_scalar_batch(op, B.scs, B.probs, B.n, part, kind, part2, kind2, exec_if,
                                        B.st);
  if (err != cudaSuccess) return cuda_fail(err, "batched scalar kernel");
  return UFG_OK;
}

// z = P_d r (tr: P_d^T) for every running problem, momentum-space evaluation (see solvers.cu).
// prep_r != nullptr: r is BiCGStab's direction p, first updated in place to
// p = prep_r + beta (p - omega prep_v) by the forward transform (slice_tma_prep_supported).
ufg_status wce_b(Batch& B, int prec, const void* r, void* z, bool tr,
                 const void* prep_r = nullptr, const void* prep_v = nullptr) {
  const int d = B.pc.order;
  std::vector<double> cw;
  if (!wce_series_weights(d, B.pc.euler, B.pc.euler_p, B.pc.vw_s, cw)) {
    set_error("WCE: invalid series acceleration parameters");
    return UFG_INVALID_ARG;
  }
  Arena& V = B.ar[prec];
  // in the momentum basis r is already spectral and the series accumulates straight into z
  void* const acc = B.mom ? z : V.acc;
  // order 2 in the momentum basis: the terms y0 (V.spec) and y1 (V.acc, unused there) are kept
  // and the last recurrence forms z = c0 y0 + c1 y1 + c2 y2 (no accumulator read-modify-write)
  const bool keep_terms = B.mom && d == 2;
  for (auto& g : B.groups) {
    const void* bk = prec ? (const void*)g.lat->bk32 : (const void*)g.lat->bk64;
    if (keep_terms) {
      if (!slice_m1w_supported(g.lat->nx, prec))
        return cuda_fail(cudaErrorInvalidValue, "momentum-basis WCE");
      auto recb = [&](const void* in, void* out, int mode, double coef) -> ufg_status {
        note_launches(1);
        KTimer kt(std::string("recurrence ") + (mode == 3 ? "sum3" : "out") +
                      (prec ? " f32" : " f64"),
                  B.st, batch_work(B, &g.probs, 0, (prec ? 4.0 : 8.0) * (mode == 3 ? 4 : 2)));
        cudaError_t e = launch_recurrence_batch(
            prec, in, out, bk, g.max_ntau, tr ? 1 : 0, 1.0, mode == 3 ? z : nullptr, coef, mode, 0,
            g.rtiles, g.nrtiles, B.probs, B.st, V.spec, V.acc, cw[0], cw[1]);
        if (e != cudaSuccess) return cuda_fail(e, "batched recurrence");
        return UFG_OK;
      };
      auto m1 = [&](const void* in) -> ufg_status {  // -A M1 (or M1^T) in momentum space
        SliceCall m = base_call(g.lat, FAM_INV, prec);
        m.fam = FAM_M1W;
        m.coef2 = base_call(g.lat, FAM_FWD, prec).coef;
        m.in = in;
        m.pre = fldb(B, 's', prec);
        if (tr) m.bkpre = bk; else m.bkpost = bk;
        m.shift = tr ? +1 : -1;
        m.a = -1.0;
        m.scale_by_A = 1;
        m.out = V.wr;
        return slice(B, g, m, 0);
      };
      UFG_TRY(recb(r, V.spec, 0, 0.0));     // y0
      UFG_TRY(m1(V.spec));
      UFG_TRY(recb(V.wr, V.acc, 0, 0.0));   // y1
      UFG_TRY(m1(V.acc));
      UFG_TRY(recb(V.wr, nullptr, 3, cw[2]));  // z = c0 y0 + c1 y1 + c2 y2
      continue;
    }
    auto rec = [&](const void* in, double coef, int mode, bool write_out) -> ufg_status {
      note_launches(1);
      KTimer kt(std::string("recurrence acc") + std::to_string(mode) + (write_out ? "+out" : "") +
                    (prec ? " f32" : " f64"),
                B.st,
                batch_work(B, &g.probs, 0,
                           (prec ? 4.0 : 8.0) *
                               (1 + (mode == 1 ? 1 : mode == 2 ? 2 : 0) + (write_out ? 1 : 0))));
      cudaError_t e = launch_recurrence_batch(prec, in, write_out ? V.spec : nullptr, bk,
                                              g.max_ntau, tr ? 1 : 0, 1.0, acc, coef, mode, 0,
                                              g.rtiles, g.nrtiles, B.probs, B.st);
      if (e != cudaSuccess) return cuda_fail(e, "batched recurrence");
      return UFG_OK;
    };
    if (B.mom) {
      UFG_TRY(rec(r, cw[0], 1, d > 0));
    } else {
      SliceCall fw = base_call(g.lat, FAM_FWD, prec);
      fw.in = r;
      fw.out = V.spec;
      if (prep_r != nullptr) {
        fw.prep_r = prep_r;
        fw.prep_v = prep_v;
        fw.prep_out = const_cast<void*>(r);
      }
      UFG_TRY(slice(B, g, fw, 0));
      UFG_TRY(rec(V.spec, cw[0], 1, d > 0));
    }
    const bool fused = slice_m1w_supported(g.lat->nx, prec);
    if (B.mom && !fused) return cuda_fail(cudaErrorInvalidValue, "momentum-basis WCE");
    for (int nn = 1; nn <= d; ++nn) {
      if (fused) {  // -A M1 (or M1^T) in momentum space in one kernel: spec -> wr
        SliceCall m = base_call(g.lat, FAM_INV, prec);
        m.fam = FAM_M1W;
        m.coef2 = base_call(g.lat, FAM_FWD, prec).coef;
        m.in = V.spec;
        m.pre = fldb(B, 's', prec);
        if (tr) m.bkpre = bk; else m.bkpost = bk;
        m.shift = tr ? +1 : -1;
        m.a = -1.0;
        m.scale_by_A = 1;
        m.out = V.wr;
        UFG_TRY(slice(B, g, m, 0));
      } else if (!tr) {
        SliceCall iv = base_call(g.lat, FAM_INV, prec);
        iv.in = V.spec;
        iv.out = V.wr;
        UFG_TRY(slice(B, g, iv, 0));
        SliceCall m1 = base_call(g.lat, FAM_FWD, prec);
        m1.in = V.wr;
        m1.pre = fldb(B, 's', prec);
        m1.bkpost = bk;
        m1.shift = -1;
        m1.a = -1.0;
        m1.scale_by_A = 1;
        m1.out = V.spec;
        UFG_TRY(slice(B, g, m1, 0));
      } else {
        SliceCall m1t = base_call(g.lat, FAM_INV, prec);
        m1t.in = V.spec;
        m1t.bkpre = bk;
        m1t.post = fldb(B, 's', prec);
        m1t.shift = +1;
        m1t.a = -1.0;
        m1t.scale_by_A = 1;
        m1t.out = V.wr;
        UFG_TRY(slice(B, g, m1t, 0));
        SliceCall fw2 = base_call(g.lat, FAM_FWD, prec);
        fw2.in = V.wr;
        fw2.out = V.spec;
        UFG_TRY(slice(B, g, fw2, 0));
      }
      UFG_TRY(rec(fused ? V.wr : V.spec, cw[nn], 2, nn < d));
    }
    if (!B.mom) {
      SliceCall iv = base_call(g.lat, FAM_INV, prec);
      iv.in = V.acc;
      iv.out = z;
      UFG_TRY(slice(B, g, iv, 0));
    }
  }
  return UFG_OK;
}

ufg_status read_scs(Batch& B) {
  UFG_CUDA(cudaMemcpyAsync(B.scs_h, B.scs, B.n * sizeof(DevScalars), cudaMemcpyDeviceToHost, B.st));
  UFG_CUDA(cudaStreamSynchronize(B.st));
  return UFG_OK;
}
ufg_status write_scs(Batch& B) {
  UFG_CUDA(cudaMemcpyAsync(B.scs, B.scs_h, B.n * sizeof(DevScalars), cudaMemcpyHostToDevice, B.st));
  return UFG_OK;
}

struct BRes {
  std::vector<int> iters, restarts, done;
};

// BiCGStab on A x = rhs for every problem whose scalars say running (tol set per problem by the
// caller in scs_h before the call); prec selects the arena.
// hook (optional): called at every host check with the scalars just read; it may act on the
// problems (e.g. replace residuals) and sets *changed when the scalars must be read again.
using CheckHook = std::function<ufg_status(bool* changed)>;

ufg_status bicg_b(Batch& B, int prec, int op, const std::vector<double>& tol,
                  const std::vector<char>& active, int maxit, int check_every, BRes* res,
                  double div_limit = 0.0, const CheckHook* hook = nullptr) {
  Arena& V = B.ar[prec];
  const bool pc = B.pc_kind == UFG_PC_WCE;
  const bool tr = op == BOP_MDAG;
  // the direction update rides on the preconditioner's first forward transform where every
  // group runs it on the TMA kernel
  bool fuse_p = pc && !B.mom;
  for (auto& g : B.groups)
    fuse_p = fuse_p && slice_tma_prep_supported(g.lat->nx, prec, g.lat->use_tma[prec]);
  for (int p = 0; p < B.n; ++p) {
    DevScalars& h = B.scs_h[p];
    std::memset(&h, 0, sizeof(DevScalars));
    h.tol = tol[p];
    h.maxit = maxit;
    h.restart_cos = 1e-12;
    h.div_limit = div_limit;
    h.rho_old = h.alpha = h.omega = 1.0;
    h.done = active[p] ? 0 : 1;
  }
  UFG_TRY(write_scs(B));
  auto init = [&](int ex, bool from_x) -> ufg_status {
    if (from_x) {
      UFG_TRY(apply_b(B, prec, op, V.x, V.r, -1.0, V.rhs, 1.0, nullptr, false, nullptr, ex));
    } else {
      UFG_TRY(vecb(B, prec, V_COPY, ex, V.r, V.rhs, nullptr, nullptr, nullptr, nullptr, nullptr));
      UFG_TRY(vecb(B, prec, V_ZERO, ex, V.x, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr));
    }
    UFG_TRY(vecb(B, prec, V_COPY, ex, V.rhat, V.r, nullptr, nullptr, nullptr, nullptr, nullptr));
    UFG_TRY(vecb(B, prec, V_ZERO, ex, V.v, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr));
    UFG_TRY(vecb(B, prec, V_ZERO, ex, V.p, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr));
    UFG_TRY(vecb(B, prec, V_DOT, ex, V.rhat, V.r, V.r, V.r, nullptr, nullptr, B.slot(B_VEC2)));
    UFG_TRY(vecb(B, prec, V_DOT, ex, V.rhat, V.rhat, V.rhs, V.rhs, nullptr, nullptr,
                 B.slot(B_DOT)));
    // with the first iteration's rho (later ones come with each iteration's residual check)
    UFG_TRY(scalb(B, OP_BI_INIT_RHO, B.slot(B_VEC2), 1, B.slot(B_DOT), 1, ex));
    return UFG_OK;
  };
  UFG_TRY(init(0, false));
  // Each scalar step is applied by the last CTA of the kernel that produces its partials.
  auto body = [&]() -> ufg_status {
    if (!fuse_p)
      UFG_TRY(vecb(B, prec, V_BI_P, 0, V.p, V.r, V.v, nullptr, nullptr, nullptr, nullptr));
    const void* y = V.p;
    if (pc) {
      UFG_TRY(wce_b(B, prec, V.p, V.y, tr, fuse_p ? V.r : nullptr, V.v));
      y = V.y;
    }
    UFG_TRY(apply_b(B, prec, op, y, V.v, 1.0, nullptr, 0.0, V.rhat, false, B.slot(B_SLICE1), 0,
                    OP_BI_ALPHA));
    UFG_TRY(vecb(B, prec, V_BI_S, 0, V.s, V.r, V.v, V.x, y, nullptr, B.slot(B_VEC1),
                 OP_BI_SCHECK));
    const void* z = V.s;
    if (pc) {
      UFG_TRY(wce_b(B, prec, V.s, V.z, tr));
      z = V.z;
    }
    UFG_TRY(apply_b(B, prec, op, z, V.t, 1.0, nullptr, 0.0, V.s, true, B.slot(B_SLICE2), 0,
                    OP_BI_OMEGA));
    UFG_TRY(vecb(B, prec, V_BI_X, 0, V.x, z, V.r, V.s, V.t, V.rhat, B.slot(B_VEC2),
                 OP_BI_RCHECK_RHO));
    return UFG_OK;
  };
  char key[192];
  snprintf(key, sizeof(key), "bicg|%d|%d|%d|%d|%d|%d|%.17g|%.17g|%d", prec, op, check_every,
           B.pc_kind, B.pc.order, B.pc.euler, B.pc.euler_p, B.pc.vw_s, B.mom ? 1 : 0);
  std::vector<int> restarts(B.n, 0);
  while (true) {
    UFG_TRY(read_scs(B));
    bool any_run = false, any_restart = false;
    for (int p = 0; p < B.n; ++p) {
      if (B.scs_h[p].done == 0) any_run = true;
      if (B.scs_h[p].done == 2) {
        if (restarts[p] < 100) {
          any_restart = true;
          ++restarts[p];
        } else {
          B.scs_h[p].done = 3;  // breakdown persisted
          UFG_CUDA(cudaMemcpyAsync(&B.scs[p].done, &B.scs_h[p].done, sizeof(int),
                                   cudaMemcpyHostToDevice, B.st));
        }
      }
    }
    if (any_restart) {
      UFG_TRY(init(2, true));
      continue;
    }
    if (hook != nullptr) {
      bool changed = false;
      UFG_TRY((*hook)(&changed));
      if (changed) continue;
    }
    if (!any_run) break;
    if (!graphs_enabled()) {
      for (int i = 0; i < check_every; ++i) UFG_TRY(body());
      continue;
    }
    // instrumented runs replay their own graphs, which carry the kernel timer's event nodes
    const std::string gkey = profiling() ? std::string(key) + "|prof" : std::string(key);
    auto it = B.graphs.find(gkey);
    if (it == B.graphs.end()) {
      const long long l0 = launches_so_far();
      profile_capture_begin();
      UFG_CUDA(cudaStreamBeginCapture(B.st, cudaStreamCaptureModeThreadLocal));
      ufg_status s = UFG_OK;
      for (int i = 0; i < check_every && s == UFG_OK; ++i) s = body();
      cudaGraph_t gr = nullptr;
      cudaError_t e = cudaStreamEndCapture(B.st, &gr);
      const long long captured = launches_so_far() - l0;
      note_launches(-captured);
      if (s != UFG_OK) {
        if (gr) cudaGraphDestroy(gr);
        profile_capture_end(nullptr);
        return s;
      }
      if (e != cudaSuccess) {
        profile_capture_end(nullptr);
        return cuda_fail(e, "cudaStreamEndCapture (batch)");
      }
      cudaGraphExec_t ex = nullptr;
      e = cudaGraphInstantiate(&ex, gr, 0);
      cudaGraphDestroy(gr);
      profile_capture_end(e == cudaSuccess ? ex : nullptr);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate (batch)");
      it = B.graphs.emplace(gkey, ex).first;
      B.graph_kernels[gkey] = captured;
    }
    UFG_CUDA(cudaGraphLaunch(it->second, B.st));
    note_launches(B.graph_kernels[gkey]);
    profile_after_replay(it->second, B.st);
  }
  res->iters.assign(B.n, 0);
  res->restarts = restarts;
  res->done.assign(B.n, 0);
  for (int p = 0; p < B.n; ++p) {
    res->iters[p] = B.scs_h[p].iters;
    res->done[p] = B.scs_h[p].done;
  }
  return UFG_OK;
}

// per-problem norms of an FP64 arena vector (host result)
ufg_status norms_b(Batch& B, const double* v, std::vector<double>& out) {
  UFG_TRY(vecb(B, 0, V_DOT, -1, nullptr, nullptr, v, v, nullptr, nullptr, B.slot(B_RES)));
  note_launches(1);
  KTimer kt("scalar", B.st, LaunchWork{});
  cudaError_t e = launch_scalar_batch(OP_NORM2, B.scs, B.probs, B.n, B.slot(B_RES), 1, nullptr, 1,
                                      -1, B.st);
  if (e != cudaSuccess) return cuda_fail(e, "batched norms");
  UFG_TRY(read_scs(B));
  out.resize(B.n);
  for (int p = 0; p < B.n; ++p) out[p] = std::sqrt(B.scs_h[p].rr);
  return UFG_OK;
}

// mode 0: y32 = s x64; mode 1: x64 += s y32; mode 2 (the fold of a reliable update, n
// problems): with s = scale[p], x64 += s y32, or with s = scale[n + p], d64 = s y32 and
// x64 += d64; y32 = 0 either way.  Problems with zero scales are skipped.
__global__ void mixed_batch_kernel(const int4* tiles, const double* scale, double* x64, float* y32,
                                   int mode, double* d64, int n) {
  pdl_begin();
  const int4 tl = tiles[blockIdx.x];
  const double sc = scale[tl.x];
  const double sd = mode == 2 ? scale[n + tl.x] : 0.0;
  if (sc == 0.0 && sd == 0.0) return;  // problem not selected
  for (long long i = (long long)tl.y + threadIdx.x; i < (long long)tl.y + tl.z; i += blockDim.x) {
    if (mode == 0) {
      y32[i] = (float)(sc * x64[i]);
    } else if (mode == 1) {
      x64[i] += sc * (double)y32[i];
    } else {
      const double v = (double)y32[i];
      if (sd != 0.0) {
        const double d = sd * v;
        d64[i] = d;
        x64[i] += d;
      } else {
        x64[i] += sc * v;
      }
      y32[i] = 0.0f;
    }
  }
}

__global__ void axpy_batch_kernel(const int4* tiles, const double* scale, double* x,
                                  const double* y, int copy) {
  pdl_begin();
  const int4 tl = tiles[blockIdx.x];
  const double sc = scale[tl.x];
  if (sc == 0.0) return;
  for (long long i = (long long)tl.y + threadIdx.x; i < (long long)tl.y + tl.z; i += blockDim.x)
    x[i] = copy ? y[i] : x[i] + sc * y[i];
}

// x += scale_p * y per problem (copy: x = y where scale_p != 0), FP64 arenas
ufg_status axpy_b(Batch& B, double* x, const double* y, const std::vector<double>& sc,
                  int copy = 0) {
  std::memcpy(B.scale_h, sc.data(), B.n * sizeof(double));
  UFG_CUDA(cudaMemcpyAsync(B.scale, B.scale_h, B.n * sizeof(double), cudaMemcpyHostToDevice, B.st));
  note_launches(1);
  KTimer kt("batch axpy f64", B.st, batch_work(B, nullptr, -1, copy ? 16.0 : 24.0));
  UFG_CUDA(launch_k(axpy_batch_kernel, dim3(B.nvtiles), dim3(256), 0, B.st, 1,
                    (const int4*)B.vtiles, (const double*)B.scale, x, y, copy));
  return UFG_OK;
}

// mode 2 takes the second scale set sd (see mixed_batch_kernel) and writes d64
ufg_status mixed_glue(Batch& B, int mode, double* x64, float* y32, const std::vector<double>& sc,
                      const std::vector<double>* sd = nullptr, double* d64 = nullptr) {
  if (mode == 2 && (sd == nullptr || d64 == nullptr)) {
    set_error("mixed glue: the fold needs the increment buffer");
    return UFG_INTERNAL;
  }
  std::memcpy(B.scale_h, sc.data(), B.n * sizeof(double));
  if (mode == 2) std::memcpy(B.scale_h + B.n, sd->data(), B.n * sizeof(double));
  const size_t nb = (mode == 2 ? 2 : 1) * (size_t)B.n * sizeof(double);
  UFG_CUDA(cudaMemcpyAsync(B.scale, B.scale_h, nb, cudaMemcpyHostToDevice, B.st));
  note_launches(1);
  KTimer kt("batch mixed glue", B.st,
            batch_work(B, nullptr, -1, mode == 0 ? 12.0 : mode == 1 ? 20.0 : 32.0));
  UFG_CUDA(launch_k(mixed_batch_kernel, dim3(B.nvtiles), dim3(256), 0, B.st, 1,
                    (const int4*)B.vtiles, (const double*)B.scale, x64, y32, mode, d64, B.n));
  return UFG_OK;
}

// Solves A x = rhs (FP64 arenas, in the batch's current basis) for every problem to per-problem
// relative tolerances.
ufg_status solve_in_basis(Batch& B, int op, const double* rhs, double* x,
                          const std::vector<double>& tol, const std::vector<char>& want,
                          const ufg_params* p, std::vector<int>& iters, std::vector<int>& outer,
                          std::vector<int>& restarts, std::vector<int>& done) {
  const size_t bytes = (size_t)B.S * sizeof(double);
  const int ce = p->check_every > 0 ? p->check_every : 8;
  std::vector<char> active = want;
  // FP64 Krylov from x = 0 for the problems in `mask`; results copied into x for those only
  auto fp64 = [&](const std::vector<char>& mask) -> ufg_status {
    Arena& V = B.ar[0];
    UFG_CUDA(cudaMemcpyAsync(V.rhs, rhs, bytes, cudaMemcpyDeviceToDevice, B.st));
    BRes r;
    UFG_TRY(bicg_b(B, 0, op, tol, mask, p->maxit, ce, &r));
    std::vector<double> sel(B.n, 0.0);
    for (int i = 0; i < B.n; ++i) {
      if (!mask[i]) continue;
      sel[i] = 1.0;
      iters[i] += r.iters[i];
      restarts[i] += r.restarts[i];
      done[i] = r.done[i];
    }
    return axpy_b(B, x, (const double*)V.x, sel, 1);
  };
  if (p->precision != UFG_MIXED) return fp64(want);
  // Mixed precision with reliable updates: one FP32 BiCGStab per problem on rhs / ||rhs||, whose
  // FP32 solution x32 is an increment to the FP64 solution x.  When a problem's recursive
  // residual has fallen by RU_DELTA since its last update (or has met the target), the
  // increment is folded into x (x += ||rhs|| x32, x32 = 0), the true residual b - A x is
  // recomputed in FP64, and the solve either stops (true residual within tol) or continues
  // from that residual without a restart: r and the restart right-hand side are replaced, the
  // search directions kept, rho and beta recomputed.
  constexpr double RU_DELTA = 1e-2;
  constexpr int RU_BUSY = 7;  // solver flag of the problems inside an update
  // FP32 too coarse for the problem: the true residual stops following the recursive one.  After
  // RU_STALLS consecutive updates that do not halve it, or RU_MAX updates, the problem is
  // finished in FP64.
  constexpr int RU_STALLS = 3, RU_MAX = 60;
  // A problem whose FP32 recursion needs more than RU_SPAN iterations for one RU_DELTA drop
  // (about four times the usual) is handed to the FP64 solver too: the batch waits for its
  // slowest problem, and a stalled FP32 Krylov space can take several times the FP64 iteration
  // count.
  constexpr int RU_SPAN = 60;
  // Incremental reliable updates (momentum basis): after a problem's first update r holds its
  // FP64 true residual, and a later update x += d (d = ||rhs|| x32) needs only
  // r -= A d, computed by the double-float operator (slice_df.cuh) on the FP32 pipe.  Its error,
  // about 2^-46 ||A|| ||d||, scales with the increment (||d|| ~ ||A^-1|| ||r||), not with x,
  // so it stays far below the residual it corrects; the first update of each solve and the
  // final residual of every problem are FP64.
  constexpr int RU_INC = 8;  // solver flag of the problems inside an incremental update
  std::vector<char> have_r(B.n, 0);
  std::vector<char> fallback(B.n, 0), verified(B.n, 0);
  std::vector<int> stalls(B.n, 0), it_last(B.n, 0);
  std::vector<double> rlast(B.n, 0.0);
  std::vector<double> bn;
  UFG_TRY(norms_b(B, rhs, bn));
  UFG_CUDA(cudaMemsetAsync(x, 0, bytes, B.st));
  Arena& V = B.ar[1];
  std::vector<double> inv(B.n, 0.0), rmax(B.n, 1.0), tin(B.n, 1.0);
  bool any = false;
  for (int i = 0; i < B.n; ++i) {
    active[i] = 0;
    if (!want[i]) continue;
    if (!std::isfinite(bn[i])) {
      done[i] = 4;
      continue;
    }
    if (bn[i] == 0.0) {
      done[i] = 1;
      continue;
    }
    active[i] = 1;
    any = true;
    inv[i] = 1.0 / bn[i];
    tin[i] = tol[i];
    outer[i] = 1;
    rlast[i] = bn[i];
  }
  if (!any) return UFG_OK;
  UFG_TRY(mixed_glue(B, 0, const_cast<double*>(rhs), (float*)V.rhs, inv));  // mode 0 reads only
  std::vector<double> rn;
  CheckHook hook = [&](bool* changed) -> ufg_status {
    *changed = false;
    bool stalled = false;
    for (int i = 0; i < B.n; ++i) {
      if (!active[i] || verified[i]) continue;
      DevScalars& h = B.scs_h[i];
      if (h.done == 0 && h.iters - it_last[i] > RU_SPAN) {
        h.done = 6;  // finished in FP64 after this solve
        stalled = true;
      }
    }
    if (stalled) {
      UFG_TRY(write_scs(B));
      *changed = true;
      return UFG_OK;
    }
    std::vector<double> sc(B.n, 0.0);
    bool upd = false;
    for (int i = 0; i < B.n; ++i) {
      if (!active[i] || verified[i]) continue;
      const DevScalars& h = B.scs_h[i];
      if (h.done != 0 && h.done != 1) continue;
      const double rr = std::sqrt(std::fmax(h.rr, 0.0));
      rmax[i] = std::fmax(rmax[i], rr);
      if (h.done == 1 || rr < RU_DELTA * rmax[i]) {
        sc[i] = bn[i];
        upd = true;
      }
    }
    if (!upd) return UFG_OK;
    *changed = true;
    // fold the increments into x and clear them (incremental updates keep d = ||rhs|| x32)
    std::vector<double> sc_full(B.n, 0.0), sc_inc(B.n, 0.0);
    bool any_full = false, any_inc = false;
    for (int i = 0; i < B.n; ++i) {
      if (sc[i] == 0.0) continue;
      const bool inc = B.mom && have_r[i];
      (inc ? sc_inc : sc_full)[i] = sc[i];
      (inc ? any_inc : any_full) = true;
      B.scs_h[i].done = inc ? RU_INC : RU_BUSY;
      it_last[i] = B.scs_h[i].iters;
    }
    UFG_TRY(mixed_glue(B, 2, x, (float*)V.x, sc_full, &sc_inc, B.d64));
    UFG_TRY(write_scs(B));
    // true residual: r = rhs - A x in FP64, or r -= A d in double-float arithmetic
    if (any_full)
      UFG_TRY(apply_b(B, 0, op, x, B.r64, -1.0, rhs, 1.0, nullptr, false, nullptr, RU_BUSY));
    if (any_inc)
      UFG_TRY(apply_b(B, 0, op, B.d64, B.r64, -1.0, B.r64, 1.0, nullptr, false, nullptr, RU_INC,
                      -1, true));
    UFG_TRY(norms_b(B, B.r64, rn));  // reads the scalars back
    std::vector<double> inv2(B.n, 0.0);
    bool cont = false;
    for (int i = 0; i < B.n; ++i) {
      if (sc[i] == 0.0) continue;
      if (!std::isfinite(rn[i])) {
        B.scs_h[i].done = 4;
      } else if (rn[i] <= tol[i] * bn[i]) {
        B.scs_h[i].done = 1;
        verified[i] = 1;
      } else {
        stalls[i] = rn[i] > 0.5 * rlast[i] ? stalls[i] + 1 : 0;
        rlast[i] = rn[i];
        if (stalls[i] >= RU_STALLS || outer[i] >= RU_MAX) {
          B.scs_h[i].done = 6;  // handed to the FP64 solver after this one
          continue;
        }
        inv2[i] = 1.0 / bn[i];
        rmax[i] = rn[i] / bn[i];
        outer[i] += 1;
        cont = true;
        have_r[i] = 1;
        B.scs_h[i].done = RU_BUSY;  // the continuation below runs on RU_BUSY
      }
    }
    UFG_TRY(write_scs(B));
    if (!cont) return UFG_OK;
    // continue from the true residual: rhs32 = r = (b - A x) / ||b||, then rho and beta again
    UFG_TRY(mixed_glue(B, 0, B.r64, (float*)V.rhs, inv2));
    UFG_TRY(vecb(B, 1, V_COPY, RU_BUSY, V.r, V.rhs, nullptr, nullptr, nullptr, nullptr,
                 nullptr));
    UFG_TRY(vecb(B, 1, V_DOT, RU_BUSY, V.rhat, V.r, V.r, V.r, nullptr, nullptr,
                 B.slot(B_VEC2)));
    UFG_TRY(scalb(B, OP_BI_RHO_REDO, B.slot(B_VEC2), 1, nullptr, 1, RU_BUSY));
    return UFG_OK;
  };
  BRes r;
  UFG_TRY(bicg_b(B, 1, op, tin, active, p->maxit, ce, &r, 1e8, &hook));
  std::vector<double> sc(B.n, 0.0);
  for (int i = 0; i < B.n; ++i) {
    if (!active[i]) continue;
    iters[i] += r.iters[i];
    restarts[i] += r.restarts[i];
    if (verified[i]) {
      done[i] = 1;
    } else if (r.done[i] == 5) {  // iteration cap: keep the progress, report not converged
      sc[i] = bn[i];
      done[i] = 5;
    } else {  // diverged, non-finite or persistent breakdown: finished in FP64
      fallback[i] = 1;
    }
  }
  UFG_TRY(mixed_glue(B, 1, x, (float*)V.x, sc));
  bool any_fb = false;
  for (int i = 0; i < B.n; ++i) any_fb = any_fb || fallback[i];
  if (any_fb) UFG_TRY(fp64(fallback));
  return UFG_OK;
}

// y = F x (inverse: F^T x) per slice for every problem, FP64 arenas
ufg_status fourier_b(Batch& B, const double* x, double* y, bool inverse) {
  for (auto& g : B.groups) {
    SliceCall c = base_call(g.lat, inverse ? FAM_INV : FAM_FWD, 0);
    c.in = x;
    c.out = y;
    UFG_TRY(slice(B, g, c, -1));
  }
  return UFG_OK;
}

// Whether the batch solves in the momentum basis: with the WCE preconditioner, whose forward and
// inverse transforms it removes, and where every group has the fused momentum-space operator in
// the precisions the solve uses (UFG_NO_MOMENTUM=1 keeps the position basis).
bool momentum_basis(const Batch& B, const ufg_params* p) {
  static int env = -1;
  if (env < 0) {
    const char* e = std::getenv("UFG_NO_MOMENTUM");
    env = (e && e[0] == '1') ? 0 : 1;
  }
  if (!env || B.pc_kind != UFG_PC_WCE) return false;
  for (const auto& g : B.groups) {
    if (!slice_m1w_supported(g.lat->nx, 0)) return false;
    if (p->precision == UFG_MIXED && !slice_m1w_supported(g.lat->nx, 1)) return false;
  }
  return true;
}

// solve_in_basis in the momentum basis where it applies: rhs to F rhs, the solve, x = F^T x^.
// Problems outside `want` get x = 0 there.
ufg_status solve_b(Batch& B, int op, const double* rhs, double* x, const std::vector<double>& tol,
                   const std::vector<char>& want, const ufg_params* p, std::vector<int>& iters,
                   std::vector<int>& outer, std::vector<int>& restarts, std::vector<int>& done) {
  if (!momentum_basis(B, p))
    return solve_in_basis(B, op, rhs, x, tol, want, p, iters, outer, restarts, done);
  UFG_TRY(fourier_b(B, rhs, B.bm64, false));
  UFG_CUDA(cudaMemsetAsync(B.xm64, 0, (size_t)B.S * sizeof(double), B.st));
  B.mom = true;
  const ufg_status s = solve_in_basis(B, op, B.bm64, B.xm64, tol, want, p, iters, outer,
                                      restarts, done);
  B.mom = false;
  UFG_TRY(s);
  return fourier_b(B, B.xm64, x, true);
}

std::string signature(int n, const ufg_problem* probs) {
  std::string sig;
  char buf[96];
  for (int i = 0; i < n; ++i) {
    snprintf(buf, sizeof(buf), "%d,%d,%.17g,%.17g;", probs[i].nx, probs[i].ntau, probs[i].tau,
             probs[i].g);
    sig += buf;
  }
  return sig;
}

// Batch workspaces are kept between calls with the same problem shapes (arenas, tile tables and
// captured graphs are reused; only sigma and b are staged per call).  At most two are cached.
std::mutex g_batch_mu;
std::vector<std::pair<std::string, std::unique_ptr<Batch>>> g_batch_cache;

// Slice tiles of every group (C CTAs per tile, g.spc time slices each), the problems' CTA
// ranges and the recurrence tiles; re-uploads the problem table when it exists already.
ufg_status build_slice_tiles(Batch& B, const ufg_problem* probs) {
  // slice tiles per group (C CTAs per tile), recurrence tiles
  int cta = 0;
  for (auto& g : B.groups) {
    std::vector<BatchTile> tl;
    std::vector<int2> rt;
    const int C = g.lat->C[0];  // same cluster size for both precisions below N_x = 32
    if (g.lat->C[1] != C) g.lat->C[1] = C;
    g.lat->spc[0] = g.lat->spc[1] = g.spc;
    g.cta_base = cta;
    for (int i : g.probs) {
      BatchProb& bp = B.probs_h[i];
      const int nt = probs[i].ntau;
      bp.off = B.off[i];
      bp.ntau = nt;
      bp.V = probs[i].nx * probs[i].nx * probs[i].nx;
      bp.A = std::sqrt(2.0) * std::sqrt(std::expm1(probs[i].tau * probs[i].g));
      bp.st0 = cta + (int)tl.size() * C;
      for (int t0 = 0; t0 < nt; t0 += g.spc) tl.push_back(BatchTile{i, t0});
      bp.st1 = cta + (int)tl.size() * C;
      for (int mb = 0; mb < (bp.V + 31) / 32; ++mb) rt.push_back(make_int2(i, mb));
      g.max_ntau = std::max(g.max_ntau, nt);
    }
    g.ntiles = (int)tl.size();
    g.nrtiles = (int)rt.size();
    cta += g.ntiles * C;
    UFG_TRY(B.alloc(&g.tiles, tl.size()));
    UFG_TRY(B.alloc(&g.rtiles, rt.size()));
    UFG_CUDA(cudaMemcpy(g.tiles, tl.data(), tl.size() * sizeof(BatchTile), cudaMemcpyHostToDevice));
    UFG_CUDA(cudaMemcpy(g.rtiles, rt.data(), rt.size() * sizeof(int2), cudaMemcpyHostToDevice));
  }
  B.nslice_ctas = cta;
  if (B.probs != nullptr)
    UFG_CUDA(cudaMemcpy(B.probs, B.probs_h.data(), B.n * sizeof(BatchProb),
                        cudaMemcpyHostToDevice));
  return UFG_OK;
}

// Time slices per slice tile, tuned per (N_x, tau) group whose slice kernels are the
// shared-memory ones in both precisions (no TMA shape at this N_x; the TMA kernels take one
// slice per CTA): at N_x = 6 a one-slice tile keeps 36 of 256 threads busy in a pass.  Each
// candidate (1, 2, 4, 8 slices within 48 KB of FP64 shared memory and the group's longest
// N_tau) is timed on the batch's own arenas with the M apply in both precisions (zeroed
// operands, three launches each after one), and the fastest is kept (ufg_stats.tile_slices).
ufg_status tune_tiles(Batch& B, const ufg_problem* probs) {
  auto tma_shape = [](int N, int prec) { return prec ? (N == 16 || N == 32) : (N == 8 || N == 16); };
  bool changed = false, zeroed = false;
  cudaEvent_t e0, e1;
  UFG_CUDA(cudaEventCreate(&e0));
  UFG_CUDA(cudaEventCreate(&e1));
  ufg_status result = UFG_OK;
  for (auto& g : B.groups) {
    const int N = g.lat->nx;
    if (tma_shape(N, 0) || tma_shape(N, 1)) continue;
    std::vector<int> cand;
    for (int spc : {1, 2, 4, 8}) {
      const size_t smem = (size_t)spc * N * (N + 1) * N * sizeof(double);
      if (spc > 1 && (smem > 48 * 1024 || spc > g.max_ntau)) break;
      cand.push_back(spc);
    }
    if (cand.size() < 2) continue;
    if (!zeroed) {
      const size_t S = (size_t)B.S;
      for (int prec = 0; prec < 2; ++prec) {
        const size_t es = prec ? sizeof(float) : sizeof(double);
        if (cudaMemsetAsync(B.ar[prec].x, 0, S * es, B.st) != cudaSuccess ||
            cudaMemsetAsync(const_cast<void*>(fldb(B, 'w', prec)), 0, S * es, B.st) !=
                cudaSuccess) {
          result = cuda_fail(cudaGetLastError(), "tile tuning");
          break;
        }
      }
      zeroed = true;
    }
    double best = 1e30;
    int best_spc = 1;
    for (int spc : cand) {
      g.spc = spc;
      if ((result = build_slice_tiles(B, probs)) != UFG_OK) break;
      float total = 0.0f;
      for (int prec = 0; prec < 2 && result == UFG_OK; ++prec) {
        SliceCall c = base_call(g.lat, FAM_KIN, prec);
        c.in = B.ar[prec].x;
        c.pre = fldb(B, 'w', prec);
        c.id = c.in;
        c.shift = -1;
        c.out = B.ar[prec].t;
        if ((result = slice(B, g, c, -1)) != UFG_OK) break;  // warm-up
        cudaEventRecord(e0, B.st);
        for (int r = 0; r < 3 && result == UFG_OK; ++r) result = slice(B, g, c, -1);
        cudaEventRecord(e1, B.st);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
          result = cuda_fail(cudaGetLastError(), "tile tuning");
          break;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        total += ms;
      }
      if (result != UFG_OK) break;
      if (total < best) {
        best = total;
        best_spc = spc;
      }
    }
    if (result != UFG_OK) break;
    g.spc = best_spc;
    changed = true;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  UFG_TRY(result);
  if (changed) UFG_TRY(build_slice_tiles(B, probs));
  return UFG_OK;
}

ufg_status setup(Batch& B, int n, const ufg_problem* probs) {
  B.n = n;
  B.pr.assign(probs, probs + n);
  UFG_CUDA(cudaStreamCreateWithFlags(&B.st, cudaStreamNonBlocking));
  // order problems by size (largest first) inside the arenas and tile tables
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return (long long)probs[a].nx * probs[a].nx * probs[a].nx * probs[a].ntau >
           (long long)probs[b].nx * probs[b].nx * probs[b].nx * probs[b].ntau;
  });
  // arena offsets padded to 256 elements: every problem starts on a row of the TMA views
  B.off.assign(n, 0);
  long long o = 0;
  for (int i : order) {
    B.off[i] = o;
    o += (long long)probs[i].nx * probs[i].nx * probs[i].nx * probs[i].ntau;
    o = (o + 255) / 256 * 256;
  }
  B.S = o;
  // groups by (N_x, tau)
  B.group_of.assign(n, -1);
  for (int i : order) {
    int gi = -1;
    for (size_t k = 0; k < B.groups.size(); ++k)
      if (B.groups[k].lat->nx == probs[i].nx && B.groups[k].lat->tau == probs[i].tau) gi = (int)k;
    if (gi < 0) {
      Group g;
      ufg_status s = ufg_lattice_create(probs[i].nx, 3, probs[i].tau, probs[i].g, 0, &g.lat);
      if (s != UFG_OK) return s;
      g.lat->spc[0] = g.lat->spc[1] = 1;
      B.groups.push_back(g);
      gi = (int)B.groups.size() - 1;
    }
    B.groups[gi].probs.push_back(i);
    B.group_of[i] = gi;
  }
  B.probs_h.assign(n, BatchProb{});
  UFG_TRY(B.alloc(&B.scs, (size_t)n));
  UFG_TRY(B.alloc(&B.counters, (size_t)n));
  UFG_CUDA(cudaMemset(B.counters, 0, n * sizeof(unsigned)));
  if (cudaMallocHost(&B.scs_h, n * sizeof(DevScalars)) != cudaSuccess ||
      cudaMallocHost(&B.scale_h, 2 * n * sizeof(double)) != cudaSuccess) {
    set_error("pinned allocation failed");
    return UFG_OOM;
  }
  UFG_TRY(B.alloc(&B.scale, 2 * (size_t)n));
  UFG_TRY(build_slice_tiles(B, probs));
  // vector tiles over the packed arenas, in arena order
  std::vector<int4> vt;
  for (int i : order) {
    BatchProb& bp = B.probs_h[i];
    const long long S = (long long)bp.V * bp.ntau;
    bp.vt0 = (int)vt.size();
    for (long long s0 = 0; s0 < S; s0 += VT_LEN)
      vt.push_back(make_int4(i, (int)(bp.off + s0), (int)std::min<long long>(VT_LEN, S - s0), 0));
    bp.vt1 = (int)vt.size();
  }
  B.nvtiles = (int)vt.size();
  UFG_TRY(B.alloc(&B.vtiles, vt.size()));
  UFG_CUDA(cudaMemcpy(B.vtiles, vt.data(), vt.size() * sizeof(int4), cudaMemcpyHostToDevice));
  for (int i = 0; i < n; ++i) B.probs_h[i].done = &B.scs[i].done;
  UFG_TRY(B.alloc(&B.probs, (size_t)n));
  UFG_CUDA(cudaMemcpy(B.probs, B.probs_h.data(), n * sizeof(BatchProb), cudaMemcpyHostToDevice));
  // partial slots
  B.part_stride = 2 * (size_t)std::max(B.nslice_ctas, B.nvtiles);
  UFG_TRY(B.alloc(&B.parts, B.part_stride * B_NSLOT));
  UFG_CUDA(cudaMemset(B.parts, 0, B.part_stride * B_NSLOT * sizeof(double)));
  // arenas and fields
  const size_t S = (size_t)B.S;
  for (int prec = 0; prec < 2; ++prec) {
    Arena& V = B.ar[prec];
    void** all[] = {&V.r, &V.rhat, &V.p, &V.v, &V.s, &V.t, &V.y, &V.z, &V.spec, &V.wr, &V.acc,
                    &V.x, &V.rhs};
    for (void** pp : all) {
      if (prec == 0) UFG_TRY(B.alloc((double**)pp, S));
      else UFG_TRY(B.alloc((float**)pp, S));
    }
  }
  UFG_TRY(B.alloc(&B.w64, S));
  UFG_TRY(B.alloc(&B.s64, S));
  UFG_TRY(B.alloc(&B.c64, S));
  UFG_TRY(B.alloc(&B.w32, S));
  UFG_TRY(B.alloc(&B.s32, S));
  UFG_TRY(B.alloc(&B.c32, S));
  UFG_TRY(B.alloc(&B.x64, S));
  UFG_TRY(B.alloc(&B.b64, S));
  UFG_TRY(B.alloc(&B.r64, S));
  UFG_TRY(B.alloc(&B.y64, S));
  UFG_TRY(B.alloc(&B.rc64, S));
  UFG_TRY(B.alloc(&B.cr64, S));
  UFG_TRY(B.alloc(&B.xm64, S));
  UFG_TRY(B.alloc(&B.bm64, S));
  UFG_TRY(B.alloc(&B.d64, S));
  return tune_tiles(B, probs);
}

// Per call: potentials from each problem's sigma and its right-hand side into the arenas.
ufg_status stage_inputs(Batch& B, const ufg_problem* probs) {
  const int n = B.n;
  for (int i = 0; i < n; ++i) {
    const BatchProb& bp = B.probs_h[i];
    const long long Sp = (long long)bp.V * bp.ntau;
    UFG_CUDA(cudaMemcpyAsync(B.y64 + bp.off, probs[i].sigma, Sp * sizeof(double),
                             cudaMemcpyDefault, B.st));
    UFG_CUDA(launch_potentials(B.y64 + bp.off, bp.A, Sp, B.w64 + bp.off, B.s64 + bp.off,
                               B.c64 + bp.off, B.w32 + bp.off, B.s32 + bp.off, B.c32 + bp.off,
                               B.st));
    note_launches(1);
    UFG_CUDA(cudaMemcpyAsync(B.b64 + bp.off, probs[i].b, Sp * sizeof(double), cudaMemcpyDefault,
                             B.st));
  }
  return UFG_OK;
}

}  // namespace

extern "C" ufg_status ufg_solve_batch(int n, const ufg_problem* probs, int pc_kind,
                                      const ufg_pc_params* pc, const ufg_params* p,
                                      ufg_stats* stats, void* stream) {
  clear_error();
  if (n <= 0 || !probs || !p || !(p->tol > 0) || p->maxit <= 0 ||
      (p->precision != UFG_FP64 && p->precision != UFG_MIXED) ||
      (pc_kind != UFG_PC_NONE && pc_kind != UFG_PC_WCE) || (pc_kind == UFG_PC_WCE && !pc)) {
    set_error("solve_batch: need n > 0, problems, params with tol > 0, maxit > 0, precision "
              "FP64 or MIXED, and preconditioner none or WCE");
    return UFG_INVALID_ARG;
  }
  for (int i = 0; i < n; ++i) {
    const ufg_problem& q = probs[i];
    if (!q.sigma || !q.b || !q.x || q.nx < 4 || q.nx % 2 || !slice_supported_n(q.nx) ||
        q.nx >= 32 || q.ntau < 3 || q.ntau > 512 || !(q.tau > 0) || !(q.g >= 0)) {
      set_error("solve_batch: problem %d invalid or unsupported (batched N_x in {4..16} built, "
                "3 <= N_tau <= 512)", i);
      return UFG_INVALID_ARG;
    }
  }
  ufg_pc_params pcn = {};
  if (pc_kind == UFG_PC_WCE) UFG_TRY(normalize_pc(pc_kind, pc, &pcn));
  const auto t0 = std::chrono::steady_clock::now();
  std::lock_guard<std::mutex> lk(g_batch_mu);
  const std::string sig = signature(n, probs);
  Batch* Bp = nullptr;
  for (auto& kv : g_batch_cache)
    if (kv.first == sig) Bp = kv.second.get();
  if (Bp == nullptr) {
    auto nb = std::make_unique<Batch>();
    ufg_status s = setup(*nb, n, probs);
    if (s != UFG_OK) return s;
    if (g_batch_cache.size() >= 2) g_batch_cache.erase(g_batch_cache.begin());
    g_batch_cache.emplace_back(sig, std::move(nb));
    Bp = g_batch_cache.back().second.get();
  }
  Batch* B = Bp;
  B->pc_kind = pc_kind;
  if (pc_kind == UFG_PC_WCE) B->pc = pcn;
  cudaStream_t user = as_stream(stream);
  cudaEvent_t ev;
  UFG_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  UFG_CUDA(cudaEventRecord(ev, user));
  UFG_CUDA(cudaStreamWaitEvent(B->st, ev, 0));
  UFG_TRY(stage_inputs(*B, probs));
  std::vector<int> it1(n, 0), it2(n, 0), out1(n, 0), out2(n, 0), rs1(n, 0), rs2(n, 0),
      d1(n, 0), d2(n, 0);
  // two-step solve of M^T M x = rhs for the problems in `want`, relative tolerance tol_i
  auto two_step = [&](const double* rhs, double* xout, const std::vector<double>& tol,
                      const std::vector<char>& want) -> ufg_status {
    std::vector<double> tol1(n), bnr, ynr, tol2(n);
    for (int i = 0; i < n; ++i) tol1[i] = 0.5 * tol[i];
    UFG_TRY(solve_b(*B, BOP_MDAG, rhs, B->y64, tol1, want, p, it1, out1, rs1, d1));
    UFG_TRY(norms_b(*B, rhs, bnr));
    UFG_TRY(norms_b(*B, B->y64, ynr));
    for (int i = 0; i < n; ++i) {
      const double A = B->probs_h[i].A;
      tol2[i] = ynr[i] > 0 ? tol[i] * bnr[i] / (2.0 * (2.0 + A) * ynr[i]) : 1.0;
    }
    return solve_b(*B, BOP_M, B->y64, xout, tol2, want, p, it2, out2, rs2, d2);
  };
  // true residual of the normal equations per problem: r = b - M^T (M x)
  std::vector<double> bn, rn;
  UFG_TRY(norms_b(*B, B->b64, bn));
  auto residual = [&]() -> ufg_status {
    for (int i = 0; i < n; ++i) B->scs_h[i].done = 0;
    UFG_TRY(write_scs(*B));
    UFG_TRY(apply_b(*B, 0, BOP_M, B->x64, B->ar[0].t, 1.0, nullptr, 0.0, nullptr, false, nullptr,
                    -1));
    UFG_TRY(apply_b(*B, 0, BOP_MDAG, B->ar[0].t, B->r64, -1.0, B->b64, 1.0, nullptr, false,
                    nullptr, -1));
    return norms_b(*B, B->r64, rn);
  };
  std::vector<char> all(n, 1);
  UFG_TRY(two_step(B->b64, B->x64, std::vector<double>(n, p->tol), all));
  UFG_TRY(residual());
  // one defect-correction round on the composite residual where it is still above tol
  std::vector<char> need(n, 0);
  std::vector<double> tolc(n, 1.0), add(n, 0.0);
  bool any = false;
  for (int i = 0; i < n; ++i) {
    if (d1[i] == 1 && d2[i] == 1 && bn[i] > 0 && rn[i] > p->tol * bn[i]) {
      need[i] = 1;
      tolc[i] = p->tol * bn[i] / rn[i];
      add[i] = 1.0;
      any = true;
    }
  }
  if (any) {
    const size_t bytes = (size_t)B->S * sizeof(double);
    UFG_CUDA(cudaMemcpyAsync(B->rc64, B->r64, bytes, cudaMemcpyDeviceToDevice, B->st));
    UFG_TRY(two_step(B->rc64, B->cr64, tolc, need));
    UFG_TRY(axpy_b(*B, B->x64, B->cr64, add));
    UFG_TRY(residual());
  }
  ufg_status worst = UFG_OK;
  for (int i = 0; i < n; ++i) {
    const BatchProb& bp = B->probs_h[i];
    const long long Sp = (long long)bp.V * bp.ntau;
    UFG_CUDA(cudaMemcpyAsync(probs[i].x, B->x64 + bp.off, Sp * sizeof(double), cudaMemcpyDefault,
                             B->st));
  }
  UFG_CUDA(cudaStreamSynchronize(B->st));
  // a bounded device wait that ran out in any group invalidates the whole batch
  ufg_status flagged = UFG_OK;
  for (auto& g : B->groups) {
    const ufg_status fs = check_device_flag(g.lat, B->st);
    if (fs != UFG_OK && flagged == UFG_OK) flagged = fs;
  }
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  for (int i = 0; i < n; ++i) {
    const int dn = (d1[i] == 1 && d2[i] == 1) ? 1 : (d1[i] != 1 ? d1[i] : d2[i]);
    ufg_status st = dn == 1 ? UFG_OK
                    : dn == 3 ? UFG_BREAKDOWN
                    : dn == 4 ? UFG_NONFINITE
                              : UFG_NOT_CONVERGED;
    const double rel = bn[i] > 0 ? rn[i] / bn[i] : 0.0;
    if (st == UFG_OK && rel > p->tol) st = UFG_NOT_CONVERGED;
    if (flagged != UFG_OK) st = flagged;
    if (st != UFG_OK && worst == UFG_OK) worst = st;
    if (stats) {
      ufg_stats& s = stats[i];
      std::memset(&s, 0, sizeof(s));
      s.status = st;
      s.iterations = it1[i] + it2[i];
      s.iterations_step[0] = it1[i];
      s.iterations_step[1] = it2[i];
      s.outer_iterations = out1[i] + out2[i];
      s.restarts = rs1[i] + rs2[i];
      const int d = pc_kind == UFG_PC_WCE ? B->pc.order : -1;
      s.n_Mdag = 2LL * it1[i];
      s.n_M = 2LL * it2[i];
      if (d >= 0) {
        s.n_M0invT = 2LL * it1[i] * (d + 1);
        s.n_M1T = 2LL * it1[i] * d;
        s.n_M0inv = 2LL * it2[i] * (d + 1);
        s.n_M1 = 2LL * it2[i] * d;
        s.mv_paper = s.iterations * 2.0 * (d + 1) * 3.0;
      } else {
        s.mv_paper = s.iterations * 2.0;
      }
      s.true_residual = rel;
      s.seconds = secs;
      s.tile_slices = B->groups[B->group_of[i]].spc;
    }
  }
  cudaEventRecord(ev, B->st);
  cudaStreamWaitEvent(user, ev, 0);
  cudaEventDestroy(ev);
  if (flagged != UFG_OK) {
    set_error("a bounded device wait ran out during the batched solve; its results are invalid");
  } else if (worst != UFG_OK) {
    set_error("at least one problem of the batch did not converge");
  }
  return worst;
}

extern "C" void ufg_batch_cache_clear(void) {
  std::lock_guard<std::mutex> lk(g_batch_mu);
  g_batch_cache.clear();
}
