// C ABI of the block-coupled solver (bcs.h). Argument checks, host/device
// staging, the Alg. 1 call sequence (structure once, values every
// iteration with full setup or values-only resetup, solve), statistics.
#include <chrono>
#include <cstdio>
#include <cmath>
#include <new>

#include "internal.h"

namespace bcs {

const char* kind_name(int k) {
  static const char* names[K_NKINDS] = {"ldu_to_bsr", "spmv_fp64",   "jacobi_sweep", "residual",
                                        "transfer",   "coarse_solve", "blas1",       "setup_aggregation",
                                        "setup_galerkin", "setup_inverse", "cast",   "scan_sort",
                                        "autotune",   "assembly"};
  return (k >= 0 && k < K_NKINDS) ? names[k] : "";
}

// Every buffer gets 16 bytes of tail padding so that 16-byte-aligned bulk
// copies of any span of it stay inside the allocation.
void* Alloc::get(size_t bytes) {
  void* p = nullptr;
  if (fa) {
    p = fa(bytes + 16, (void*)stream, user);
    if (p && reinterpret_cast<uintptr_t>(p) % 256 != 0) {
      // the kernels use 16-byte vector accesses and rely on 256-byte bases
      fr(p, bytes + 16, (void*)stream, user);
      return nullptr;
    }
    if (p) live += bytes;
    return p;
  }
  if (cudaMallocAsync(&p, bytes + 16, stream) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  live += bytes;
  return p;
}

void Alloc::put(void* p, size_t bytes) {
  if (!p) return;
  if (fr) fr(p, bytes + 16, (void*)stream, user);
  else (void)cudaFreeAsync(p, stream);
  live -= bytes;
}

void Solver::pre(int kind) {
  if (!cfg.profile || (cfg.profile_kinds && !(cfg.profile_kinds & (1 << kind)))) return;
  if (event_next + 2 > event_pool.size()) {
    for (int q = 0; q < 64; ++q) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return;
      event_pool.push_back(e);
    }
  }
  Timer t{kind, event_pool[event_next], event_pool[event_next + 1], nullptr, 0.0, cur_level};
  event_next += 2;
  cudaEventRecord(t.a, stream);
  timers.push_back(t);
}

bcs_status Solver::post(int kind, const char* what, double bytes, double flops) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(BCS_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
  ++launches;
  kind_launches[kind]++;
  kind_bytes[kind] += bytes;
  kind_flops[kind] += flops;
  if (cfg.profile && !timers.empty() && timers.back().kind == kind && !timers.back().what) {
    cudaEventRecord(timers.back().b, stream);
    timers.back().what = what;
    timers.back().bytes = bytes;
  }
  return BCS_OK;
}

void Solver::flush_timers() {
  if (timers.empty()) return;
  cudaStreamSynchronize(stream);
  for (const Timer& t : timers) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) {
      kind_ms[t.kind] += ms;
      if (t.level >= 0 && t.level < LEVEL_TIMES_MAX) {
        if ((int)level_times.size() <= t.level) level_times.resize(t.level + 1);
        LevelTime& lt = level_times[t.level];
        lt.launches[t.kind]++;
        lt.ms[t.kind] += ms;
        lt.bytes[t.kind] += t.bytes;
      }
      if (t.what) {
        NamedTime& nt = named[t.what];
        nt.launches++;
        nt.ms += ms;
        nt.bytes += t.bytes;
        nt.kind = t.kind;
      }
    }
  }
  timers.clear();
  event_next = 0;
}

}  // namespace bcs

using namespace bcs;

namespace {

bcs_status check_config(const bcs_config* c) {
  if (c->solver != BCS_FGMRES && c->solver != BCS_BICGSTAB) return BCS_EINVAL;
  if (c->restart < 1 || c->restart > 64) return BCS_EINVAL;
  if (!(c->tol > 0.0) || c->maxiter < 1) return BCS_EINVAL;
  if (c->precond < BCS_PC_AMG || c->precond > BCS_PC_SGS) return BCS_EINVAL;
  if (c->pmode != BCS_P_SMOOTHED && c->pmode != BCS_P_TENTATIVE) return BCS_EINVAL;
  if (c->matching_rounds < 1 || c->agg_passes < 1 || c->agg_passes > 4) return BCS_EINVAL;
  if (c->nu1 < 0 || c->nu2 < 0 || c->nu1 + c->nu2 < 1) return BCS_EINVAL;
  if (c->coarse_size < 1 || c->max_levels < 1 || c->coarse_sweeps < 1) return BCS_EINVAL;
  if (c->coarse_dense_max < 1 || c->coarse_dense_max > 8192) return BCS_EINVAL;
  if (c->precision < BCS_PREC_FP64 || c->precision > BCS_PREC_BF16) return BCS_EINVAL;
  if (c->cycle_graph < -1 || c->cycle_graph > 1) return BCS_EINVAL;
  if (c->reorder < 0 || c->reorder > 1) return BCS_EINVAL;
  if (c->tail_rows < 0) return BCS_EINVAL;
  if (c->dilu_cluster_rows < 0) return BCS_EINVAL;
  if (c->dependent_launch < 0 || c->dependent_launch > 1) return BCS_EINVAL;
  if (c->x0_zero < 0 || c->x0_zero > 1) return BCS_EINVAL;
  if ((c->alloc == nullptr) != (c->release == nullptr)) return BCS_EINVAL;
  if (c->slice_layout < -1 || c->slice_layout > 1) return BCS_EINVAL;
  if (c->smoother < BCS_SMOOTH_JACOBI || c->smoother > BCS_SMOOTH_SGS) return BCS_EINVAL;
  if (!(c->max_coarsen_ratio > 0.0) || !(c->p_omega > 0.0) || !(c->jacobi_omega > 0.0)) return BCS_EINVAL;
  return BCS_OK;
}

bool same_hierarchy_options(const bcs_config& a, const bcs_config& b) {
  return a.precond == b.precond && a.pmode == b.pmode && a.matching_rounds == b.matching_rounds &&
         a.agg_passes == b.agg_passes && a.jacobi_omega == b.jacobi_omega && a.nu1 == b.nu1 && a.nu2 == b.nu2 &&
         a.coarse_size == b.coarse_size && a.max_levels == b.max_levels &&
         a.max_coarsen_ratio == b.max_coarsen_ratio && a.p_omega == b.p_omega &&
         a.coarse_dense_max == b.coarse_dense_max && a.coarse_sweeps == b.coarse_sweeps &&
         a.precision == b.precision && a.slice_layout == b.slice_layout &&
         a.smoother == b.smoother;
}

// Copy a host array into a device staging buffer (or pass a device pointer).
template <class T>
bcs_status stage(Solver* s, const T* src, size_t count, int mem, DBuf<T>& buf, const T** out) {
  if (mem == BCS_MEM_DEVICE || count == 0) {
    *out = src;
    if (count == 0 && !src) *out = nullptr;
    return BCS_OK;
  }
  BCS_ALLOC(s, buf, count);
  BCS_CU(s, cudaMemcpyAsync(buf.p, src, count * sizeof(T), cudaMemcpyHostToDevice, s->stream));
  *out = buf.p;
  return BCS_OK;
}

double ms_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

bcs_status to_host(Solver* s, void* dst, const void* src, size_t bytes) {
  if (!dst || bytes == 0) return BCS_OK;
  BCS_CU(s, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s->stream));
  BCS_CU(s, cudaStreamSynchronize(s->stream));
  return BCS_OK;
}

// After new fine values: full AMG setup, or values-only resetup.
bcs_status values_changed(Solver* s, std::chrono::steady_clock::time_point t0) {
  struct DirectCopyDone {  // a gather's sliced copy belongs to these values only
    Solver* s;
    ~DirectCopyDone() { s->v0_direct = -1; }
  } done{s};
  s->have_values = true;
  const bool full = !s->have_hierarchy;
  if (full) s->setup_cfg = s->cfg;
  s->have_hierarchy = false;
  BCS_OKR(amg_setup(s, full));
  // a values-only resetup rewrites every buffer in place (same sizes, same
  // addresses), so the captured cycle and Krylov graphs stay valid
  BCS_OKR(cycle_prepare(s, !full));
  BCS_CU(s, cudaStreamSynchronize(s->stream));
  s->have_hierarchy = true;
  s->last_setup_ms = ms_since(t0);
  return BCS_OK;
}

}  // namespace

extern "C" {

bcs_status bcs_config_default(bcs_config* c) {
  if (!c) return BCS_EINVAL;
  std::memset(c, 0, sizeof(*c));
  c->solver = BCS_FGMRES;
  c->restart = 30;
  c->tol = 1e-8;
  c->maxiter = 1000;
  c->precond = BCS_PC_AMG;
  c->pmode = BCS_P_TENTATIVE;
  c->matching_rounds = 4;
  c->agg_passes = 2;
  c->jacobi_omega = 0.8;
  c->nu1 = 2;
  c->nu2 = 2;
  c->coarse_size = 32;
  c->max_levels = 20;
  c->max_coarsen_ratio = 0.8;
  c->p_omega = 4.0 / 3.0;
  c->coarse_dense_max = 1024;
  c->coarse_sweeps = 8;
  c->precision = BCS_PREC_FP32;
  c->profile = 0;
  c->profile_kinds = 0;
  c->smoother = BCS_SMOOTH_JACOBI;
  c->slice_layout = -1;
  c->cycle_graph = -1;
  c->reorder = 0;
  c->tail_rows = 0;
  c->dilu_cluster_rows = 4096;
  c->dependent_launch = 1;
  c->x0_zero = 0;
  return BCS_OK;
}

bcs_status bcs_create(bcs_solver** out, int n, const bcs_config* cfg, void* stream) {
  if (!out) return BCS_EINVAL;
  *out = nullptr;
  if (n < 1 || n > 8) return BCS_EINVAL;
  bcs_config c;
  if (cfg) c = *cfg;
  else bcs_config_default(&c);
  if (check_config(&c) != BCS_OK) return BCS_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return BCS_ECUDA;
  }
  // Keep freed blocks in the stream-ordered pool instead of returning them
  // at every synchronisation (setup allocates and frees temporaries).
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  bcs_solver* h = new (std::nothrow) bcs_solver();
  if (!h) return BCS_ENOMEM;
  Solver* s = &h->impl;
  s->n = n;
  s->cfg = c;
  s->setup_cfg = c;
  s->stream = (cudaStream_t)stream;
  s->alloc.stream = s->stream;
  s->alloc.fa = c.alloc;
  s->alloc.fr = c.release;
  s->alloc.user = c.alloc_user;
  if (!s->flag.resize(&s->alloc, 4) || !s->scal.resize(&s->alloc, 160) ||
      cudaMallocHost(&s->hscal, 160 * sizeof(double)) != cudaSuccess) {
    (void)cudaGetLastError();
    delete h;
    return BCS_ENOMEM;
  }
  if (cudaMemsetAsync(s->flag.p, 0, 4 * sizeof(int32_t), s->stream) != cudaSuccess) {
    delete h;
    return BCS_ECUDA;
  }
  *out = h;
  return BCS_OK;
}

bcs_status bcs_destroy(bcs_solver* h) {
  if (!h) return BCS_OK;
  Solver* s = &h->impl;
  cudaStreamSynchronize(s->stream);
  s->drop_graph();
  if (s->gstream) cudaStreamDestroy(s->gstream);
  if (s->cstream) {
    cudaStreamSynchronize(s->cstream);
    cudaStreamDestroy(s->cstream);
  }
  if (s->sstream) {
    cudaStreamSynchronize(s->sstream);
    cudaStreamDestroy(s->sstream);
  }
  for (cudaEvent_t e : s->sev)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : s->copy_events) cudaEventDestroy(e);
  for (cudaEvent_t e : s->event_pool) cudaEventDestroy(e);
  if (s->hscal) cudaFreeHost(s->hscal);
  cudaStream_t st = s->stream;
  delete h;  // frees device buffers (stream-ordered)
  cudaStreamSynchronize(st);
  return BCS_OK;
}

bcs_status bcs_set_config(bcs_solver* h, const bcs_config* cfg) {
  if (!h || !cfg) return BCS_EINVAL;
  Solver* s = &h->impl;
  if (check_config(cfg) != BCS_OK) return s->fail(BCS_EINVAL, "invalid configuration");
  if (!same_hierarchy_options(*cfg, s->setup_cfg)) s->have_hierarchy = false;
  s->cfg = *cfg;
  return BCS_OK;
}

bcs_status bcs_set_structure(bcs_solver* h, int32_t C, int32_t F, const int32_t* owner, const int32_t* nb,
                             int mem) {
  NvtxRange nvtx_("bcs_set_structure");
  if (!h) return BCS_EINVAL;
  Solver* s = &h->impl;
  s->have_structure = s->have_values = s->have_hierarchy = false;
  if (C < 1 || F < 0 || (F > 0 && (!owner || !nb)) || (mem != BCS_MEM_HOST && mem != BCS_MEM_DEVICE))
    return s->fail(BCS_EINVAL, "invalid structure arguments");
  s->C = C;
  s->F = F;
  const int32_t *o = nullptr, *m = nullptr;
  BCS_OKR(stage(s, owner, (size_t)F, mem, s->stage_o, &o));
  BCS_OKR(stage(s, nb, (size_t)F, mem, s->stage_n, &m));
  s->reordered = false;
  s->perm.release();
  s->inv.release();
  bcs_status st = build_structure(s, o, m);
  if (st == BCS_OK && s->cfg.reorder == 1) {
    // reverse Cuthill-McKee on the caller's numbering, then the structure
    // again with relabelled faces; face blocks keep their LDU slots
    BCS_ALLOC(s, s->perm, C);
    BCS_ALLOC(s, s->inv, C);
    st = rcm_order(s, s->lv[0].A, s->perm.p, s->inv.p);
    DBuf<int32_t> o2, m2;
    if (st == BCS_OK && F > 0) {
      BCS_ALLOC(s, o2, F);
      BCS_ALLOC(s, m2, F);
      st = relabel_faces(s, o, m, o2.p, m2.p);
    }
    if (st == BCS_OK) st = build_structure(s, o2.p, m2.p);
    if (st == BCS_OK) st = user_diag_maps(s);
    if (st == BCS_OK) s->reordered = true;
  }
  s->stage_o.release();
  s->stage_n.release();
  if (st != BCS_OK) return st;
  BCS_CU(s, cudaStreamSynchronize(s->stream));
  s->have_structure = true;
  return BCS_OK;
}

bcs_status bcs_set_values(bcs_solver* h, const double* diag, const double* upper, const double* lower, int mem) {
  NvtxRange nvtx_("bcs_set_values");
  if (!h) return BCS_EINVAL;
  Solver* s = &h->impl;
  if (!s->have_structure) return s->fail(BCS_ESTATE, "set_values before set_structure");
  if (!diag || (s->F > 0 && (!upper || !lower)) || (mem != BCS_MEM_HOST && mem != BCS_MEM_DEVICE))
    return s->fail(BCS_EINVAL, "invalid value arguments");
  const auto t0 = std::chrono::steady_clock::now();
  if (mem == BCS_MEM_HOST) {
    BCS_OKR(upload_values(s, diag, upper, lower));
    return values_changed(s, t0);
  }
  BCS_OKR(permute_values(s, diag, upper, lower));
  return values_changed(s, t0);
}

bcs_status bcs_flow_params_default(bcs_flow_params* p) {
  if (!p) return BCS_EINVAL;
  p->gamma = 1.4;
  p->mu = 1e-3;
  p->prandtl = 0.72;
  p->cfl = 10.0;
  return BCS_OK;
}

bcs_status bcs_assemble_density(bcs_solver* h, const double* Q, const double* area, const double* normal,
                                const double* dist, const bcs_flow_params* prm, double* diag, double* upper,
                                double* lower, int mem) {
  NvtxRange nvtx_("bcs_assemble_density");
  if (!h) return BCS_EINVAL;
  Solver* s = &h->impl;
  if (!s->have_structure) return s->fail(BCS_ESTATE, "assemble before set_structure");
  if (s->n != 5) return s->fail(BCS_EINVAL, "the density-based assembly needs 5x5 blocks");
  const bool to_values = !diag && !upper && !lower;
  if (!prm || !Q || (s->F > 0 && (!area || !normal || !dist)) || (mem != BCS_MEM_HOST && mem != BCS_MEM_DEVICE) ||
      (!to_values && (!diag || (s->F > 0 && (!upper || !lower)))))
    return s->fail(BCS_EINVAL, "invalid assembly arguments");
  if (!(prm->gamma > 1.0) || !(prm->mu >= 0.0) || !(prm->prandtl > 0.0) || !(prm->cfl > 0.0) ||
      !std::isfinite(prm->gamma) || !std::isfinite(prm->mu) || !std::isfinite(prm->prandtl) ||
      !std::isfinite(prm->cfl))
    return s->fail(BCS_EINVAL, "invalid flow parameters");
  const auto t0 = std::chrono::steady_clock::now();
  const size_t C = s->C, F = s->F;
  const double *q = nullptr, *a = nullptr, *nv = nullptr, *d = nullptr;
  DBuf<double> sq, sa, sn, sd, od, ou, ol;
  BCS_OKR(stage(s, Q, C * 5, mem, sq, &q));
  BCS_OKR(stage(s, area, F, mem, sa, &a));
  BCS_OKR(stage(s, normal, F * 3, mem, sn, &nv));
  BCS_OKR(stage(s, dist, F, mem, sd, &d));
  if (to_values) {
    // the fine values are replaced: on failure the solver has no values and
    // no hierarchy until the next successful upload
    s->have_values = false;
    const bool had = s->have_hierarchy;
    s->have_hierarchy = false;
    BCS_OKR(assemble_density(s, q, a, nv, d, *prm, nullptr, nullptr, nullptr));
    s->have_hierarchy = had;
    return values_changed(s, t0);
  }
  double *dd = diag, *du = upper, *dl = lower;
  if (mem == BCS_MEM_HOST) {
    BCS_ALLOC(s, od, C * 25);
    BCS_ALLOC(s, ou, F > 0 ? F * 25 : 1);
    BCS_ALLOC(s, ol, F > 0 ? F * 25 : 1);
    dd = od.p;
    du = ou.p;
    dl = ol.p;
  }
  BCS_OKR(assemble_density(s, q, a, nv, d, *prm, dd, du, dl));
  if (mem == BCS_MEM_HOST) {
    BCS_OKR(to_host(s, diag, dd, C * 25 * sizeof(double)));
    BCS_OKR(to_host(s, upper, du, F * 25 * sizeof(double)));
    BCS_OKR(to_host(s, lower, dl, F * 25 * sizeof(double)));
  }
  return BCS_OK;
}

static bcs_status check_fields(Solver* s, int nfields, const int* ncomp, int mem) {
  if (!s->have_structure) return s->fail(BCS_ESTATE, "field conversion before set_structure");
  if (nfields < 1 || nfields > PK_MAX_FIELDS || !ncomp || (mem != BCS_MEM_HOST && mem != BCS_MEM_DEVICE))
    return s->fail(BCS_EINVAL, "invalid field arguments");
  int n = 0;
  for (int k = 0; k < nfields; ++k) {
    if (ncomp[k] < 1) return s->fail(BCS_EINVAL, "a field with no components");
    n += ncomp[k];
  }
  if (n != s->n) return s->fail(BCS_EINVAL, "field components do not add up to the block size");
  return BCS_OK;
}

bcs_status bcs_pack_vector(bcs_solver* h, int nfields, const int* ncomp, const double* const* fields, double* out,
                           int mem) {
  NvtxRange nvtx_("bcs_pack_vector");
  if (!h) return BCS_EINVAL;
  Solver* s = &h->impl;
  BCS_OKR(check_fields(s, nfields, ncomp, mem));
  if (!fields || !out) return s->fail(BCS_EINVAL, "null field array");
  for (int k = 0; k < nfields; ++k)
    if (!fields[k]) return s->fail(BCS_EINVAL, "null field array");
  const size_t C = s->C;
  DBuf<double> st[PK_MAX_FIELDS], o;
  const double* in[PK_MAX_FIELDS] = {};
  for (int k = 0; k < nfields; ++k) BCS_OKR(stage(s, fields[k], C * ncomp[k], mem, st[k], &in[k]));
  double* od = out;
  if (mem == BCS_MEM_HOST) {
    BCS_ALLOC(s, o, C * s->n);
    od = o.p;
  }
  BCS_OKR(pack_vector(s, nfields, ncomp, in, od));
  if (mem == BCS_MEM_HOST) return to_host(s, out, od, C * s->n * sizeof(double));
  BCS_CU(s, cudaStreamSynchronize(s->stream));
  return BCS_OK;
}

bcs_status bcs_unpack_vector(bcs_solver* h, int nfields, const int* ncomp, const double* in, double* const* fields,
                             int mem) {
  NvtxRange nvtx_("bcs_unpack_vector");
  if (!h) return BCS_EINVAL;
  Solver* s = &h->impl;
  BCS_OKR(check_fields(s, nfields, ncomp, mem));
  if (!fields || !in) return s->fail(BCS_EINVAL, "null field array");
  for (int k = 0; k < nfields; ++k)
    if (!fields[k]) return s->fail(BCS_EINVAL, "null field array");
  const size_t C = s->C;
  DBuf<double> si, so[PK_MAX_FIELDS];
  const double* ind = nullptr;
  BCS_OKR(stage(s, in, C * s->n, mem, si, &ind));
  double* outs[PK_MAX_FIELDS] = {};
  for (int k = 0; k < nfields; ++k) {
    outs[k] = fields[k];
    if (mem == BCS_MEM_HOST) {
      BCS_ALLOC(s, so[k], C * ncomp[k]);
      outs[k] = so[k].p;
    }
  }
  BCS_OKR(unpack_vector(s, nfields, ncomp, ind, outs));
  if (mem == BCS_MEM_HOST)
    for (int k = 0; k < nfields; ++k) BCS_OKR(to_host(s, fields[k], outs[k], C * ncomp[k] * sizeof(double)));
  BCS_CU(s, cudaStreamSynchronize(s->stream));
  return BCS_OK;
}

bcs_status bcs_pack_coefficients(bcs_solver* h, int nfields, const int* ncomp, const bcs_coupling* coupling,
                                 double* diag, double* upper, double* lower, int mem) {
  NvtxRange nvtx_("bcs_pack_coefficients");
  if (!h) return BCS_EINVAL;
  Solver* s = &h->impl;
  BCS_OKR(check_fields(s, nfields, ncomp, mem));
  const bool to_values = !diag && !upper && !lower;
  if (!coupling || (!to_values && (!diag || (s->F > 0 && (!upper || !lower)))))
    return s->fail(BCS_EINVAL, "invalid coefficient arguments");
  const auto t0 = std::chrono::steady_clock::now();
  const size_t C = s->C, F = s->F;
  std::vector<DBuf<double>> st(3 * nfields * nfields);
  std::vector<const double*> src(3 * nfields * nfields, nullptr);
  for (int a = 0; a < nfields; ++a)
    for (int b = 0; b < nfields; ++b) {
      const int p = a * nfields + b;
      const bcs_coupling& cp = coupling[p];
      const bool none = !cp.diag && !cp.upper && !cp.lower;
      if (none) continue;
      if (!cp.diag || (F > 0 && (!cp.upper || !cp.lower)))
        return s->fail(BCS_EINVAL, "a coupling with only some of its arrays");
      const size_t m = (size_t)ncomp[a] * ncomp[b];
      BCS_OKR(stage(s, cp.diag, C * m, mem, st[3 * p], &src[3 * p]));
      BCS_OKR(stage(s, cp.upper, F * m, mem, st[3 * p + 1], &src[3 * p + 1]));
      BCS_OKR(stage(s, cp.lower, F * m, mem, st[3 * p + 2], &src[3 * p + 2]));
    }
  if (to_values) {
    s->have_values = false;
    const bool had = s->have_hierarchy;
    s->have_hierarchy = false;
    BCS_OKR(pack_coefficients(s, nfields, ncomp, src.data(), nullptr, nullptr, nullptr));
    s->have_hierarchy = had;
    return values_changed(s, t0);
  }
  const size_t nn = (size_t)s->n * s->n;
  DBuf<double> od, ou, ol;
  double *dd = diag, *du = upper, *dl = lower;
  if (mem == BCS_MEM_HOST) {
    BCS_ALLOC(s, od, C * nn);
    BCS_ALLOC(s, ou, F > 0 ? F * nn : 1);
    BCS_ALLOC(s, ol, F > 0 ? F * nn : 1);
    dd = od.p;
    du = ou.p;
    dl = ol.p;
  }
  BCS_OKR(pack_coefficients(s, nfields, ncomp, src.data(), dd, du, dl));
  if (mem == BCS_MEM_HOST) {
    BCS_OKR(to_host(s, diag, dd, C * nn * sizeof(double)));
    BCS_OKR(to_host(s, upper, du, F * nn * sizeof(double)));
    BCS_OKR(to_host(s, lower, dl, F * nn * sizeof(double)));
  }
  BCS_CU(s, cudaStreamSynchronize(s->stream));
  return BCS_OK;
}

bcs_status bcs_get_permutation(bcs_solver* h, int32_t* perm) {
  if (!h) return BCS_EINVAL;
  Solver* s = &h->impl;
  if (!s->have_structure) return s->fail(BCS_ESTATE, "no structure");
  if (!perm) return s->fail(BCS_EINVAL, "null permutation");
  if (!s->reordered) {
    for (int i = 0; i < s->C; ++i) perm[i] = i;
    return BCS_OK;
  }
  return to_host(s, perm, s->perm.p, (size_t)s->C * sizeof(int32_t));
}

bcs_status bcs_invalidate_hierarchy(bcs_solver* h) {
  if (!h) return BCS_EINVAL;
  h->impl.have_hierarchy = false;
  return BCS_OK;
}

bcs_status bcs_solve_batch(bcs_solver* const* solvers, int count, const double* const* b, double* const* x, int mem,
                           bcs_result* res) {
  NvtxRange nvtx_("bcs_solve_batch");
  if (!solvers || !b || !x || !res || count < 1 || count > BCS_BATCH_MAX) return BCS_EINVAL;
  if (mem != BCS_MEM_HOST && mem != BCS_MEM_DEVICE) return BCS_EINVAL;
  std::vector<Solver*> ss(count);
  for (int i = 0; i < count; ++i) {
    if (!solvers[i] || !b[i] || !x[i]) return BCS_EINVAL;
    ss[i] = &solvers[i]->impl;
    for (int k = 0; k < i; ++k)
      if (ss[k] == ss[i]) return ss[0]->fail(BCS_EINVAL, "batched solve: a solver appears twice");
  }
  Solver* s0 = ss[0];
  const bcs_config& c0 = s0->setup_cfg;
  for (int i = 0; i < count; ++i) {
    Solver* s = ss[i];
    const bcs_config& c = s->setup_cfg;
    if (!s->have_hierarchy) return s0->fail(BCS_ESTATE, "batched solve: a solver has no values yet");
    if (!same_hierarchy_options(s->cfg, s->setup_cfg))
      return s0->fail(BCS_ESTATE, "batched solve: options changed since a solver's last set_values");
    if (s->n != s0->n || s->reordered || s->cfg.solver != BCS_FGMRES || c.precond != BCS_PC_AMG ||
        c.smoother != BCS_SMOOTH_JACOBI || c.pmode != BCS_P_TENTATIVE ||
        (c.precision != BCS_PREC_FP32 && c.precision != BCS_PREC_BF16) || c.precision != c0.precision ||
        c.nu1 != c0.nu1 || c.nu2 != c0.nu2 || c.jacobi_omega != c0.jacobi_omega ||
        c.coarse_sweeps != c0.coarse_sweeps || s->cfg.restart != s0->cfg.restart || s->cfg.restart > KS_MAXM ||
        (int)s->lv.size() > BATCH_MAX_LEVELS)
      return s0->fail(BCS_EINVAL,
                      "batched solve: the solvers need the same block size, FGMRES, an FP32 or BF16 aggregation "
                      "AMG cycle with block Jacobi and tentative prolongation, the same smoothing options and "
                      "restart length, and no internal renumbering");
    if (s->cfg.profile && (s->cfg.profile_kinds == 0 || (s->cfg.profile_kinds & ~((1 << K_SETUP_AGG) |
                                                                                   (1 << K_SETUP_GAL) |
                                                                                   (1 << K_SETUP_INV) |
                                                                                   (1 << K_CONVERT) |
                                                                                   (1 << K_ASSEMBLE)))))
      return s0->fail(BCS_EINVAL, "batched solve: per-kernel events of the solve kinds cannot be taken in it");
    BCS_CU(s0, cudaStreamSynchronize(s->stream));
  }
  std::vector<const double*> bd(count);
  std::vector<double*> xd(count);
  for (int i = 0; i < count; ++i) {
    bd[i] = b[i];
    xd[i] = x[i];
    if (mem == BCS_MEM_HOST) {
      Solver* s = ss[i];
      const size_t N = (size_t)s->C * s->n;
      BCS_ALLOC(s, s->kb, N);
      BCS_ALLOC(s, s->kx, N);
      BCS_CU(s, cudaMemcpyAsync(s->kb.p, b[i], N * sizeof(double), cudaMemcpyHostToDevice, s->stream));
      if (!s->cfg.x0_zero)
        BCS_CU(s, cudaMemcpyAsync(s->kx.p, x[i], N * sizeof(double), cudaMemcpyHostToDevice, s->stream));
      BCS_CU(s, cudaStreamSynchronize(s->stream));
      bd[i] = s->kb.p;
      xd[i] = s->kx.p;
    }
    if (ss[i]->cfg.x0_zero) {
      Solver* s = ss[i];
      BCS_CU(s, cudaMemsetAsync(xd[i], 0, (size_t)s->C * s->n * sizeof(double), s->stream));
      BCS_CU(s, cudaStreamSynchronize(s->stream));
    }
  }
  BCS_OKR(solve_batch(ss.data(), count, bd.data(), xd.data(), res));
  BCS_CU(s0, cudaStreamSynchronize(s0->stream));
  bcs_status worst = BCS_OK;
  for (int i = 0; i < count; ++i) {
    if (mem == BCS_MEM_HOST) BCS_OKR(to_host(ss[i], x[i], xd[i], (size_t)ss[i]->C * ss[i]->n * sizeof(double)));
    if (res[i].status != BCS_OK && worst == BCS_OK) worst = (bcs_status)res[i].status;
  }
  return worst;
}

bcs_status bcs_solve(bcs_solver* h, const double* b, double* x, int mem, bcs_result* res) {
  NvtxRange nvtx_("bcs_solve");
  if (!h) return BCS_EINVAL;
  Solver* s = &h->impl;
  bcs_result local{};
  if (!res) res = &local;
  std::memset(res, 0, sizeof(*res));
  if (!s->have_hierarchy) return s->fail(BCS_ESTATE, "solve before set_values");
  if (!b || !x || (mem != BCS_MEM_HOST && mem != BCS_MEM_DEVICE)) return s->fail(BCS_EINVAL, "invalid solve arguments");
  if (!same_hierarchy_options(s->cfg, s->setup_cfg))
    return s->fail(BCS_ESTATE, "options changed since the last set_values");
  const size_t N = (size_t)s->C * s->n;
  const double* bd = b;
  double* xd = x;
  if (mem == BCS_MEM_HOST) {
    BCS_ALLOC(s, s->kb, N);
    BCS_ALLOC(s, s->kx, N);
    BCS_CU(s, cudaMemcpyAsync(s->kb.p, b, N * sizeof(double), cudaMemcpyHostToDevice, s->stream));
    if (!s->cfg.x0_zero)
      BCS_CU(s, cudaMemcpyAsync(s->kx.p, x, N * sizeof(double), cudaMemcpyHostToDevice, s->stream));
    bd = s->kb.p;
    xd = s->kx.p;
  }
  if (s->cfg.x0_zero) BCS_CU(s, cudaMemsetAsync(xd, 0, N * sizeof(double), s->stream));
  double* xu = xd;  // x in the caller's numbering on the device
  if (s->reordered) {
    BCS_ALLOC(s, s->rb, N);
    BCS_ALLOC(s, s->rx, N);
    BCS_OKR(to_internal(s, bd, s->rb.p));
    BCS_OKR(to_internal(s, xd, s->rx.p));
    bd = s->rb.p;
    xd = s->rx.p;
  }
  bcs_status st = solve(s, bd, xd, res);
  if (st == BCS_ECUDA || st == BCS_ENOMEM || st == BCS_EINVAL) return st;
  if (s->reordered) BCS_OKR(to_user(s, xd, xu));
  if (mem == BCS_MEM_HOST) BCS_OKR(to_host(s, x, xu, N * sizeof(double)));
  return st;
}

bcs_status bcs_spmv(bcs_solver* h, const double* x, double* y, int mem) {
  NvtxRange nvtx_("bcs_spmv");
  if (!h) return BCS_EINVAL;
  Solver* s = &h->impl;
  if (!s->have_values) return s->fail(BCS_ESTATE, "spmv before set_values");
  if (!x || !y) return s->fail(BCS_EINVAL, "null vector");
  const size_t N = (size_t)s->C * s->n;
  const double* xd = x;
  double* yd = y;
  if (mem == BCS_MEM_HOST) {
    BCS_ALLOC(s, s->kb, N);
    BCS_ALLOC(s, s->kx, N);
    BCS_CU(s, cudaMemcpyAsync(s->kb.p, x, N * sizeof(double), cudaMemcpyHostToDevice, s->stream));
    xd = s->kb.p;
    yd = s->kx.p;
  }
  if (s->reordered) {
    BCS_ALLOC(s, s->rb, N);
    BCS_ALLOC(s, s->rx, N);
    BCS_OKR(to_internal(s, xd, s->rb.p));
    BCS_OKR(spmv64(s, s->lv[0].A, s->rb.p, false, s->rx.p, nullptr, K_SPMV64));
    BCS_OKR(to_user(s, s->rx.p, yd));
  } else {
    BCS_OKR(spmv64(s, s->lv[0].A, xd, false, yd, nullptr, K_SPMV64));
  }
  if (mem == BCS_MEM_HOST) BCS_OKR(to_host(s, y, yd, N * sizeof(double)));
  BCS_CU(s, cudaStreamSynchronize(s->stream));
  return BCS_OK;
}

bcs_status bcs_precond_apply(bcs_solver* h, const double* v, double* z, int mem) {
  NvtxRange nvtx_("bcs_precond_apply");
  if (!h) return BCS_EINVAL;
  Solver* s = &h->impl;
  if (!s->have_hierarchy) return s->fail(BCS_ESTATE, "precond_apply before set_values");
  if (!v || !z) return s->fail(BCS_EINVAL, "null vector");
  const size_t N = (size_t)s->C * s->n;
  BCS_ALLOC(s, s->kb, N);
  BCS_ALLOC(s, s->kx, N);
  DBuf<char> zt;
  BCS_ALLOC(s, zt, N * sizeof(double));
  const double* vd = v;
  if (mem == BCS_MEM_HOST) {
    BCS_CU(s, cudaMemcpyAsync(s->kb.p, v, N * sizeof(double), cudaMemcpyHostToDevice, s->stream));
    vd = s->kb.p;
  }
  double* zd = mem == BCS_MEM_HOST ? s->kx.p : z;
  double* zu = zd;  // z in the caller's numbering on the device
  if (s->reordered) {
    BCS_ALLOC(s, s->rb, N);
    BCS_ALLOC(s, s->rx, N);
    BCS_OKR(to_internal(s, vd, s->rb.p));
    vd = s->rb.p;
    zd = s->rx.p;
  }
  switch (s->setup_cfg.precond) {
    case BCS_PC_AMG:
    case BCS_PC_SGS:
      BCS_OKR(s->setup_cfg.precond == BCS_PC_AMG ? precond_apply(s, vd, zt.p) : sgs_apply(s, vd, zt.p));
      if (cycle_is_float(s)) BCS_OKR(cast_vec<float, double>(s, (const float*)zt.p, zd, N));
      else BCS_CU(s, cudaMemcpyAsync(zd, zt.p, N * sizeof(double), cudaMemcpyDeviceToDevice, s->stream));
      break;
    case BCS_PC_JACOBI:
      BCS_OKR(jacobi_apply(s, vd, zd));
      break;
    default:
      BCS_CU(s, cudaMemcpyAsync(zd, vd, N * sizeof(double), cudaMemcpyDeviceToDevice, s->stream));
  }
  if (s->reordered) BCS_OKR(to_user(s, zd, zu));
  if (mem == BCS_MEM_HOST) BCS_OKR(to_host(s, z, zu, N * sizeof(double)));
  BCS_CU(s, cudaStreamSynchronize(s->stream));
  return BCS_OK;
}

bcs_status bcs_get_bsr(bcs_solver* h, int32_t* rp, int32_t* col, double* val, int32_t* pd, int32_t* pu,
                       int32_t* pl) {
  if (!h) return BCS_EINVAL;
  Solver* s = &h->impl;
  if (!s->have_structure) return s->fail(BCS_ESTATE, "no structure");
  const Bsr& A = s->lv[0].A;
  BCS_OKR(to_host(s, rp, A.rp.p, (A.rows + 1) * sizeof(int32_t)));
  BCS_OKR(to_host(s, col, A.ci.p, (size_t)A.nnz * sizeof(int32_t)));
  if (val) {
    if (!s->have_values) return s->fail(BCS_ESTATE, "no values");
    BCS_OKR(to_host(s, val, A.v.p, (size_t)A.nnz * s->n * s->n * sizeof(double)));
  }
  BCS_OKR(to_host(s, pd, s->pos_diag.p, (size_t)s->C * sizeof(int32_t)));
  BCS_OKR(to_host(s, pu, s->pos_up.p, (size_t)s->F * sizeof(int32_t)));
  BCS_OKR(to_host(s, pl, s->pos_lo.p, (size_t)s->F * sizeof(int32_t)));
  return BCS_OK;
}

int bcs_num_levels(const bcs_solver* h) {
  if (!h || !h->impl.have_hierarchy) return 0;
  return (int)h->impl.lv.size();
}

bcs_status bcs_get_level_info(const bcs_solver* h, int l, int* rows, int* nnz, int* p_nnz, int* kind) {
  if (!h) return BCS_EINVAL;
  const Solver* s = &h->impl;
  if (!s->have_hierarchy || l < 0 || l >= (int)s->lv.size()) return BCS_EINVAL;
  const Level& L = s->lv[l];
  if (rows) *rows = L.A.rows;
  if (nnz) *nnz = L.A.nnz;
  if (p_nnz) *p_nnz = (L.coarse_kind < 0 && s->setup_cfg.pmode == BCS_P_SMOOTHED) ? L.P.nnz : 0;
  if (kind) *kind = L.coarse_kind;
  return BCS_OK;
}

bcs_status bcs_get_level(bcs_solver* h, int l, int32_t* rp, int32_t* col, double* val, int32_t* agg,
                         double* dinv) {
  if (!h) return BCS_EINVAL;
  Solver* s = &h->impl;
  if (!s->have_hierarchy || l < 0 || l >= (int)s->lv.size()) return s->fail(BCS_EINVAL, "no such level");
  const Level& L = s->lv[l];
  const size_t nn = (size_t)s->n * s->n;
  BCS_OKR(to_host(s, rp, L.A.rp.p, (L.A.rows + 1) * sizeof(int32_t)));
  BCS_OKR(to_host(s, col, L.A.ci.p, (size_t)L.A.nnz * sizeof(int32_t)));
  BCS_OKR(to_host(s, val, L.A.v.p, (size_t)L.A.nnz * nn * sizeof(double)));
  if (agg && L.coarse_kind < 0) BCS_OKR(to_host(s, agg, L.agg.p, (size_t)L.A.rows * sizeof(int32_t)));
  if (dinv) {
    DBuf<double> tmp;
    const double* d64 = nullptr;
    BCS_OKR(level_dinv64(s, l, &d64, tmp));
    BCS_OKR(to_host(s, dinv, d64, (size_t)L.A.rows * nn * sizeof(double)));
  }
  return BCS_OK;
}

bcs_status bcs_get_prolongation(bcs_solver* h, int l, int32_t* rp, int32_t* col, double* val, double* omega) {
  if (!h) return BCS_EINVAL;
  Solver* s = &h->impl;
  if (!s->have_hierarchy || l < 0 || l + 1 >= (int)s->lv.size() || s->setup_cfg.pmode != BCS_P_SMOOTHED)
    return s->fail(BCS_EINVAL, "no smoothed prolongation at this level");
  const Level& L = s->lv[l];
  BCS_OKR(to_host(s, rp, L.P.rp.p, (L.P.rows + 1) * sizeof(int32_t)));
  BCS_OKR(to_host(s, col, L.P.ci.p, (size_t)L.P.nnz * sizeof(int32_t)));
  BCS_OKR(to_host(s, val, L.P.v.p, (size_t)L.P.nnz * s->n * s->n * sizeof(double)));
  if (omega) *omega = L.omega_p;
  return BCS_OK;
}

bcs_status bcs_get_coarse_inverse(bcs_solver* h, double* inv) {
  if (!h) return BCS_EINVAL;
  Solver* s = &h->impl;
  if (!s->have_hierarchy || s->lv.back().coarse_kind != 0) return s->fail(BCS_EINVAL, "no dense coarse inverse");
  return to_host(s, inv, s->cinv.p, (size_t)s->cN * s->cN * sizeof(double));
}

bcs_status bcs_get_dilu(bcs_solver* h, int level, int* ncolours, int32_t* colour, double* einv) {
  if (!h || !ncolours) return BCS_EINVAL;
  Solver* s = &h->impl;
  if (!s->have_hierarchy || level < 0 || level >= (int)s->lv.size()) return s->fail(BCS_EINVAL, "no such level");
  const Level& L = s->lv[level];
  *ncolours = L.ncol > 0 ? L.ncol : -1;
  if (L.ncol <= 0) return BCS_OK;
  if (colour) BCS_OKR(to_host(s, colour, L.colour.p, (size_t)L.A.rows * sizeof(int32_t)));
  if (einv) {
    DBuf<double> tmp;
    const double* e64 = nullptr;
    BCS_OKR(dilu_einv64(s, level, &e64, tmp));
    BCS_OKR(to_host(s, einv, e64, (size_t)L.A.rows * s->n * s->n * sizeof(double)));
  }
  return BCS_OK;
}

bcs_status bcs_get_stats(bcs_solver* h, bcs_stats* st) {
  if (!h || !st) return BCS_EINVAL;
  Solver* s = &h->impl;
  s->flush_timers();
  std::memset(st, 0, sizeof(*st));
  st->launches = s->launches;
  for (int k = 0; k < BCS_NUM_KERNEL_KINDS; ++k) {
    st->kind_launches[k] = s->kind_launches[k];
    st->kind_ms[k] = s->kind_ms[k];
    st->kind_bytes[k] = s->kind_bytes[k];
    st->kind_flops[k] = s->kind_flops[k];
  }
  return BCS_OK;
}

bcs_status bcs_get_kernel_times(bcs_solver* h, char* buf, size_t len) {
  if (!h || !buf || !len) return BCS_EINVAL;
  Solver* s = &h->impl;
  s->flush_timers();
  std::string out;
  char line[512];
  for (const auto& kv : s->named) {
    std::snprintf(line, sizeof(line), "%s\t%lld\t%.6f\t%.0f\t%d\n", kv.first.c_str(), kv.second.launches,
                  kv.second.ms, kv.second.bytes, kv.second.kind);
    out += line;
  }
  std::snprintf(buf, len, "%s", out.c_str());
  return out.size() < len ? BCS_OK : BCS_EINVAL;
}

bcs_status bcs_reset_stats(bcs_solver* h) {
  if (!h) return BCS_EINVAL;
  Solver* s = &h->impl;
  s->flush_timers();
  s->named.clear();
  s->level_times.clear();
  s->launches = 0;
  for (int k = 0; k < BCS_NUM_KERNEL_KINDS; ++k) {
    s->kind_launches[k] = 0;
    s->kind_ms[k] = 0.0;
    s->kind_bytes[k] = 0.0;
    s->kind_flops[k] = 0.0;
  }
  return BCS_OK;
}

bcs_status bcs_get_level_times(bcs_solver* h, int level, long long* launches, double* ms, double* bytes) {
  if (!h || !launches || !ms || !bytes || level < 0 || level >= LEVEL_TIMES_MAX) return BCS_EINVAL;
  Solver* s = &h->impl;
  s->flush_timers();
  const LevelTime none{};
  const LevelTime& lt = level < (int)s->level_times.size() ? s->level_times[level] : none;
  for (int k = 0; k < BCS_NUM_KERNEL_KINDS; ++k) {
    launches[k] = lt.launches[k];
    ms[k] = lt.ms[k];
    bytes[k] = lt.bytes[k];
  }
  return BCS_OK;
}

const char* bcs_kernel_kind_name(int k) { return kind_name(k); }

const char* bcs_last_error(const bcs_solver* h) { return h ? h->impl.err.c_str() : "null solver"; }

size_t bcs_device_bytes(const bcs_solver* h) { return h ? h->impl.alloc.live : 0; }

}  // extern "C"
