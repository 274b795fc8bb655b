// C ABI entry points (include/fcgle.h): argument validation, exception to
// status translation and the thread-local error message.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "engine.h"
#include "norm_static.h"
#include "selftest.h"

struct fcgle_ctx {
  fcgle_params prm;
  cudaStream_t stream = nullptr;
  std::unique_ptr<fcgle::EngineBase> eng;
  // bumped by fcgle_set_coefficients / fcgle_set_source: captured batch steps
  // carry the coefficients by value and must be rebuilt after a change
  unsigned long long gen = 0;
};

// Batch of independent instances: one stream per group of instances (longest
// processing time first on the mode-product work), a step of all instances
// captured once into a CUDA graph (fork / join over the streams) and replayed.
struct fcgle_batch_ctx {
  std::vector<fcgle_ctx*> inst;
  cudaStream_t main = nullptr;     // the caller's stream (may be the legacy default stream)
  cudaStream_t origin = nullptr;   // internal stream the step graph is captured from and launched on
  cudaEvent_t enter = nullptr, leave = nullptr;
  std::vector<cudaStream_t> streams;
  std::vector<int> stream_of;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  std::map<std::pair<int, uint64_t>, cudaGraphExec_t> graphs;
  long long graph_launches = 0;
  // grouped persistent launches: per (scheme, tau) the phases of one step,
  // each one launch over the descriptors of all instances in that phase
  struct Phase {
    void (*launch)(const void*, int, long long, cudaStream_t);
    size_t offset;     // of its descriptor array in dev
    int n;
    long long units;
    std::vector<void (*)(const void*, int, long long, cudaStream_t)> alts;   // equivalent configurations
    std::vector<std::string> alt_names;
  };
  struct Plan {
    std::vector<Phase> phases;
    void* dev = nullptr;
    cudaGraphExec_t graph = nullptr;
  };
  std::map<std::pair<int, uint64_t>, Plan> plans;
  long long grouped_kernels = 0;
  unsigned long long gen_built = 0;   // sum of the instances' gen when graphs / plans were built
};

namespace fcgle {

static thread_local std::string g_last_error;

void throw_cuda(cudaError_t e, const char* where) {
  throw CudaError{e, std::string(where) + ": " + cudaGetErrorString(e)};
}

namespace {

fcgle_status fail(fcgle_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

template <typename F>
fcgle_status guarded(F&& f) {
  try {
    g_last_error.clear();
    f();
    return FCGLE_OK;
  } catch (const InvalidArg& e) {
    return fail(FCGLE_ERR_INVALID_ARG, e.what());
  } catch (const Unsupported& e) {
    return fail(FCGLE_ERR_UNSUPPORTED, e.what());
  } catch (const NumericError& e) {
    return fail(FCGLE_ERR_NUMERIC, e.what());
  } catch (const DeviceTimeout& e) {
    return fail(FCGLE_ERR_TIMEOUT, e.what());
  } catch (const CudaError& e) {
    if (e.err == cudaErrorMemoryAllocation) return fail(FCGLE_ERR_NOMEM, e.where);
    return fail(FCGLE_ERR_CUDA, e.where);
  } catch (const std::bad_alloc&) {
    return fail(FCGLE_ERR_NOMEM, "host allocation failed");
  } catch (const std::exception& e) {
    return fail(FCGLE_ERR_CUDA, e.what());
  }
}

void validate(const fcgle_params* p) {
  if (!p) throw InvalidArg("params is NULL");
  if (p->d < 1 || p->d > 3) throw InvalidArg("d must be 1, 2 or 3");
  for (int mu = 0; mu < p->d; ++mu) {
    if (p->n[mu] < 1) throw InvalidArg("n_mu must be >= 1");
    if (p->n[mu] > 8192) throw InvalidArg("n_mu must be <= 8192");
    if (!(p->alpha[mu] > 1.0 && p->alpha[mu] < 2.0)) throw InvalidArg("alpha_mu must lie in (1, 2)");
    if (!(p->b[mu] > p->a[mu])) throw InvalidArg("b_mu must exceed a_mu");
  }
  if (!(p->nu > 0.0)) throw InvalidArg("nu must be positive");
  if (!(p->kappa > 0.0)) throw InvalidArg("kappa must be positive");
  if (!std::isfinite(p->eta) || !std::isfinite(p->gamma) || !std::isfinite(p->zeta))
    throw InvalidArg("eta, gamma, zeta must be finite");
  if (p->fd_order != 2 && p->fd_order != 4) throw InvalidArg("fd_order must be 2 or 4");
  if (p->precision == FCGLE_TF32) throw Unsupported("FCGLE_TF32 (one-pass TF32 mode products) is not built");
  if (p->precision != FCGLE_FP64 && p->precision != FCGLE_BF16X3) throw InvalidArg("unknown precision");
}

void check_handle(fcgle_handle h) {
  if (!h || !h->eng) throw InvalidArg("invalid handle");
}

void check_scheme(int scheme) {
  if (scheme < FCGLE_LIE || scheme > FCGLE_STRANG) throw InvalidArg("unknown scheme");
}

void check_tau(double tau) {
  if (!(tau > 0.0) || !std::isfinite(tau)) throw InvalidArg("tau must be positive and finite");
}

// Turns a code read from an engine's device error word into the C status.
void report_device(int code) {
  if (code == kErrNonFinite) throw NumericError("the result state holds a non-finite value (NaN or Inf)");
  if (code) throw DeviceTimeout("a bounded device-side wait gave up (code " + std::to_string(code) + ")");
}

}  // namespace
}  // namespace fcgle

using namespace fcgle;

extern "C" {

fcgle_status fcgle_setup(const fcgle_params* params, void* cuda_stream, fcgle_handle* out) {
  return guarded([&] {
    if (!out) throw InvalidArg("out is NULL");
    *out = nullptr;
    validate(params);
    auto* ctx = new fcgle_ctx;
    try {
      ctx->prm = *params;
      ctx->stream = (cudaStream_t)cuda_stream;
      ctx->eng = make_engine(*params, ctx->stream);
      ctx->eng->autotune();
    } catch (...) {
      delete ctx;
      throw;
    }
    *out = ctx;
  });
}

fcgle_status fcgle_set_stream(fcgle_handle h, void* cuda_stream) {
  return guarded([&] {
    check_handle(h);
    h->stream = (cudaStream_t)cuda_stream;
    h->eng->set_stream(h->stream);
  });
}

fcgle_status fcgle_set_source(fcgle_handle h, int nterms, const double* sigma_reim, const void* const* S_dev) {
  return guarded([&] {
    check_handle(h);
    if (nterms < 0 || nterms > kMaxSrc) throw InvalidArg("nterms must be in 0..4");
    if (nterms > 0 && (!sigma_reim || !S_dev)) throw InvalidArg("sigma_reim / S_dev is NULL");
    for (int k = 0; k < nterms; ++k) {
      if (!S_dev[k]) throw InvalidArg("source tensor is NULL");
      if (!std::isfinite(sigma_reim[2 * k]) || !std::isfinite(sigma_reim[2 * k + 1]))
        throw InvalidArg("sigma must be finite");
    }
    h->eng->set_source(nterms, sigma_reim, S_dev);
    ++h->gen;
  });
}

fcgle_status fcgle_set_coefficients(fcgle_handle h, double nu, double eta, double gamma, double kappa,
                                    double zeta) {
  return guarded([&] {
    check_handle(h);
    if (!(nu > 0.0)) throw InvalidArg("nu must be positive");
    if (!(kappa > 0.0)) throw InvalidArg("kappa must be positive");
    if (!std::isfinite(eta) || !std::isfinite(gamma) || !std::isfinite(zeta))
      throw InvalidArg("eta, gamma, zeta must be finite");
    h->eng->set_coefficients(nu, eta, gamma, kappa, zeta);
    h->prm.nu = nu;
    h->prm.eta = eta;
    h->prm.gamma = gamma;
    h->prm.kappa = kappa;
    h->prm.zeta = zeta;
    ++h->gen;
  });
}

fcgle_status fcgle_set_exp_form(fcgle_handle h, int form) {
  return guarded([&] {
    check_handle(h);
    h->eng->set_exp_form(form);
    ++h->gen;
  });
}

fcgle_status fcgle_set_tucker_form(fcgle_handle h, int form) {
  return guarded([&] {
    check_handle(h);
    h->eng->set_tucker_form(form);
    ++h->gen;
  });
}

fcgle_status fcgle_apply_f(fcgle_handle h, int func, int k, double theta, const void* v, void* out) {
  return guarded([&] {
    check_handle(h);
    if (func < FCGLE_F_INV || func > FCGLE_F_PHI) throw InvalidArg("unknown func");
    if (func == FCGLE_F_PHI && (k < 0 || k > 4)) throw InvalidArg("phi order k must be in 0..4");
    if (!std::isfinite(theta)) throw InvalidArg("theta must be finite");
    if (!v || !out) throw InvalidArg("tensor pointer is NULL");
    h->eng->apply_f(func, k, theta, v, out);
  });
}

fcgle_status fcgle_spectral_scalars(fcgle_handle h, int func, int k, double theta, int count, const double* s_host,
                                    double* out_host, int flags) {
  return guarded([&] {
    check_handle(h);
    if (func < FCGLE_F_INV || func > FCGLE_F_PHI) throw InvalidArg("unknown func");
    if (func == FCGLE_F_PHI && (k < 0 || k > 4)) throw InvalidArg("phi order k must be in 0..4");
    if (!std::isfinite(theta)) throw InvalidArg("theta must be finite");
    if (count < 0) throw InvalidArg("count must be >= 0");
    if (count > 0 && (!s_host || !out_host)) throw InvalidArg("pointer is NULL");
    for (int j = 0; j < count; ++j)
      if (!std::isfinite(s_host[j])) throw InvalidArg("eigenvalue sums must be finite");
    if (flags & ~1) throw InvalidArg("unknown flags");
    if ((flags & 1) && h->prm.precision != FCGLE_BF16X3) throw InvalidArg("the ray form needs a BF16X3 handle");
    h->eng->spectral_scalars(func, k, theta, count, s_host, out_host, flags);
  });
}

fcgle_status fcgle_step(fcgle_handle h, int scheme, double tau, double t, void* u) {
  return guarded([&] {
    check_handle(h);
    check_scheme(scheme);
    if (scheme == FCGLE_LBDF2) throw InvalidArg("LBDF2 is a two-step scheme: use fcgle_integrate");
    check_tau(tau);
    if (!u) throw InvalidArg("u is NULL");
    h->eng->step(scheme, tau, t, u);
  });
}

fcgle_status fcgle_integrate(fcgle_handle h, int scheme, double tau, int nsteps, double t0, const void* u0,
                             void* uT) {
  return guarded([&] {
    check_handle(h);
    check_scheme(scheme);
    check_tau(tau);
    if (nsteps < 0) throw InvalidArg("nsteps must be >= 0");
    if (!u0 || !uT) throw InvalidArg("tensor pointer is NULL");
    h->eng->integrate(scheme, tau, nsteps, t0, u0, uT);
  });
}

fcgle_status fcgle_integrate_host(fcgle_handle h, int scheme, double tau, int nsteps, double t0,
                                  const void* u0_host, void* uT_host) {
  return guarded([&] {
    check_handle(h);
    check_scheme(scheme);
    check_tau(tau);
    if (nsteps < 0) throw InvalidArg("nsteps must be >= 0");
    if (!u0_host || !uT_host) throw InvalidArg("tensor pointer is NULL");
    h->eng->integrate_host(scheme, tau, nsteps, t0, u0_host, uT_host);
    report_device(h->eng->device_error());
  });
}

fcgle_status fcgle_adjoint(fcgle_handle h, int scheme, double tau, int nsteps, double t0, const void* u0,
                           const void* u_target, int ckpt_every, void* grad_u0, double* grad_params, double* loss) {
  return guarded([&] {
    check_handle(h);
    check_scheme(scheme);
    check_tau(tau);
    if (nsteps < 0) throw InvalidArg("nsteps must be >= 0");
    if (ckpt_every < 0) throw InvalidArg("ckpt_every must be >= 0");
    if (!u0 || !u_target || !grad_u0 || !grad_params || !loss) throw InvalidArg("pointer is NULL");
    h->eng->adjoint(scheme, tau, nsteps, t0, u0, u_target, ckpt_every, grad_u0, grad_params, loss);
    report_device(h->eng->device_error());
    if (!std::isfinite(*loss)) throw NumericError("the misfit is not finite");
    for (int k = 0; k < 5; ++k)
      if (!std::isfinite(grad_params[k])) throw NumericError("a parameter gradient is not finite");
  });
}

fcgle_status fcgle_norm(fcgle_handle h, const void* u, double* out_host) {
  return guarded([&] {
    check_handle(h);
    if (!u || !out_host) throw InvalidArg("pointer is NULL");
    *out_host = h->eng->norm(u);
  });
}

fcgle_status fcgle_norm_static(const fcgle_params* p, const void* u, void* cuda_stream, double* out_host) {
  return guarded([&] {
    if (!p || !u || !out_host) throw InvalidArg("pointer is NULL");
    if (p->d < 1 || p->d > 3) throw InvalidArg("d must be 1, 2 or 3");
    unsigned long long N = 1;
    double cell = 1.0;
    for (int mu = 0; mu < p->d; ++mu) {
      if (p->n[mu] < 1) throw InvalidArg("n_mu must be >= 1");
      if (!(p->b[mu] > p->a[mu])) throw InvalidArg("b_mu must exceed a_mu");
      N *= (unsigned long long)p->n[mu];
      cell *= (p->b[mu] - p->a[mu]) / (p->n[mu] + 1.0);
    }
    if (p->precision != FCGLE_FP64 && p->precision != FCGLE_BF16X3) throw InvalidArg("unknown precision");
    const double s = norm_static_sumsq(u, p->precision == FCGLE_FP64, N, (cudaStream_t)cuda_stream);
    *out_host = std::sqrt(cell * s);
  });
}

fcgle_status fcgle_selftest_bounded_wait(void* cuda_stream, int* code_out) {
  return guarded([&] {
    if (!code_out) throw InvalidArg("code_out is NULL");
    *code_out = 0;
    const int code = bounded_wait_selftest((cudaStream_t)cuda_stream);
    *code_out = code;
    if (code) throw DeviceTimeout("a bounded device-side wait gave up (code " + std::to_string(code) + ")");
  });
}

fcgle_status fcgle_sync(fcgle_handle h) {
  return guarded([&] {
    check_handle(h);
    report_device(h->eng->device_error());
  });
}

fcgle_status fcgle_sizes(fcgle_handle h, size_t* n_elems, size_t* n_bytes) {
  return guarded([&] {
    check_handle(h);
    size_t N = 1;
    for (int mu = 0; mu < h->prm.d; ++mu) N *= (size_t)h->prm.n[mu];
    if (n_elems) *n_elems = N;
    if (n_bytes) *n_bytes = N * h->eng->elem_bytes();
  });
}

fcgle_status fcgle_internal_elems(fcgle_handle h, size_t* P) {
  return guarded([&] {
    check_handle(h);
    if (!P) throw InvalidArg("P is NULL");
    *P = h->eng->internal_elems();
  });
}

fcgle_status fcgle_mode_product(fcgle_handle h, int direction, int flags, const void* X, void* Y) {
  return guarded([&] {
    check_handle(h);
    if (!X || !Y) throw InvalidArg("tensor pointer is NULL");
    if (X == Y) throw InvalidArg("X and Y must not overlap");
    if (flags & ~31) throw InvalidArg("unknown flags");
    h->eng->mode_product_flags(direction, flags, X, Y);
  });
}

fcgle_status fcgle_launch_count(fcgle_handle h, long long* count) {
  return guarded([&] {
    check_handle(h);
    if (!count) throw InvalidArg("count is NULL");
    *count = h->eng->launches;
  });
}

fcgle_status fcgle_destroy(fcgle_handle h) {
  return guarded([&] {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    delete h;
  });
}

// ------------------------------------------------------------------ batches
// Drops every captured step graph and grouped plan (after the work that may
// still use them has finished).
static void batch_drop_cache(fcgle_batch_ctx* b) {
  if (b->origin) cudaStreamSynchronize(b->origin);
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
  for (auto& kv : b->plans) {
    if (kv.second.graph) cudaGraphExecDestroy(kv.second.graph);
    if (kv.second.dev) cudaFree(kv.second.dev);
  }
  b->graphs.clear();
  b->plans.clear();
}

static void batch_free(fcgle_batch_ctx* b) {
  if (!b) return;
  batch_drop_cache(b);
  for (auto* h : b->inst) delete h;
  for (auto st : b->streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  if (b->origin) cudaStreamDestroy(b->origin);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->enter) cudaEventDestroy(b->enter);
  if (b->leave) cudaEventDestroy(b->leave);
  for (auto e : b->join) cudaEventDestroy(e);
  delete b;
}

fcgle_status fcgle_batch_create(int count, const fcgle_params* params, void* cuda_stream, int nstreams,
                                fcgle_batch* out) {
  return guarded([&] {
    if (!out) throw InvalidArg("out is NULL");
    *out = nullptr;
    if (count < 1 || !params) throw InvalidArg("count must be >= 1 and params non-NULL");
    if (nstreams < 1) nstreams = std::min(count, 16);
    nstreams = std::min(nstreams, count);
    for (int i = 0; i < count; ++i) validate(&params[i]);
    auto* b = new fcgle_batch_ctx;
    try {
      b->main = (cudaStream_t)cuda_stream;
      b->streams.resize(nstreams);
      b->join.resize(nstreams);
      for (int k = 0; k < nstreams; ++k) {
        FCGLE_CUDA(cudaStreamCreateWithFlags(&b->streams[k], cudaStreamNonBlocking));
        FCGLE_CUDA(cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming));
      }
      FCGLE_CUDA(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
      FCGLE_CUDA(cudaEventCreateWithFlags(&b->enter, cudaEventDisableTiming));
      FCGLE_CUDA(cudaEventCreateWithFlags(&b->leave, cudaEventDisableTiming));
      FCGLE_CUDA(cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking));
      // longest processing time first: work of a step ~ N * sum_mu n_mu
      std::vector<std::pair<double, int>> cost(count);
      for (int i = 0; i < count; ++i) {
        double N = 1, S = 0;
        for (int mu = 0; mu < params[i].d; ++mu) {
          N *= params[i].n[mu];
          S += params[i].n[mu];
        }
        cost[i] = {N * S, i};
      }
      std::sort(cost.begin(), cost.end(), [](auto& x, auto& y) { return x.first > y.first; });
      std::vector<double> load(nstreams, 0.0);
      b->stream_of.assign(count, 0);
      for (auto& c : cost) {
        const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        b->stream_of[c.second] = k;
        load[k] += c.first;
      }
      // set the instances up in parallel host threads (the eigensolvers dominate)
      b->inst.assign(count, nullptr);
      std::vector<std::string> errs(count);
      std::atomic<int> next(0);
      const int nth = std::max(1, std::min(count, (int)std::thread::hardware_concurrency() / 2));
      std::vector<std::thread> th;
      for (int w = 0; w < nth; ++w)
        th.emplace_back([&] {
          for (int i = next++; i < count; i = next++) {
            try {
              auto* h = new fcgle_ctx;
              h->prm = params[i];
              h->stream = b->streams[b->stream_of[i]];
              h->eng = make_engine(params[i], h->stream);
              // the grouped launches run every Tucker operator in the rotating
              // form; the instances' own launches use it too, so that every path
              // of a batch rounds alike
              h->eng->set_tucker_form(FCGLE_TUCKER_ROTATING);
              b->inst[i] = h;
            } catch (const std::exception& e) {
              errs[i] = e.what();
            } catch (const CudaError& e) {
              errs[i] = e.where;
            }
          }
        });
      for (auto& t : th) t.join();
      for (int i = 0; i < count; ++i)
        if (!b->inst[i]) throw std::runtime_error("instance " + std::to_string(i) + ": " + errs[i]);
      // timing runs one instance at a time, so that no other work overlaps them
      FCGLE_CUDA(cudaDeviceSynchronize());
      for (auto* h : b->inst) h->eng->autotune();
    } catch (...) {
      batch_free(b);
      throw;
    }
    *out = b;
  });
}

fcgle_status fcgle_batch_instance(fcgle_batch b, int i, fcgle_handle* h) {
  return guarded([&] {
    if (!b || !h) throw InvalidArg("NULL argument");
    if (i < 0 || i >= (int)b->inst.size()) throw InvalidArg("instance index out of range");
    *h = b->inst[i];
  });
}

static void tune_plan(fcgle_batch_ctx::Plan& plan, cudaStream_t st);

// Record step `n` of every instance and group the records into phases: for
// each Tucker operator of the step, the k-th inner mode product of all
// instances (k = 0, 1, ..), then the last mode products; records of one phase
// with the same kernel type share a launch.  Returns false (nothing built) if
// an instance has no grouped form.
static bool build_plan(fcgle_batch_ctx* b, int n, cudaStream_t st, fcgle_batch_ctx::Plan& plan) {
  const int ni = (int)b->inst.size();
  std::vector<std::vector<fcgle::GroupRec>> recs(ni);
  bool ok = true;
  for (int i = 0; i < ni && ok; ++i) {
    if (!b->inst[i]->eng->set_recorder(&recs[i])) {
      ok = false;
      break;
    }
    try {
      b->inst[i]->eng->one_step(n);
    } catch (...) {
      b->inst[i]->eng->set_recorder(nullptr);
      throw;
    }
    b->inst[i]->eng->set_recorder(nullptr);
  }
  if (!ok) return false;
  // split each instance's records into Tucker operators (each ends with a `last` record)
  std::vector<std::vector<std::vector<const fcgle::GroupRec*>>> tk(ni);
  for (int i = 0; i < ni; ++i) {
    std::vector<const fcgle::GroupRec*> cur;
    for (const auto& r : recs[i]) {
      cur.push_back(&r);
      if (r.last) {
        tk[i].push_back(cur);
        cur.clear();
      }
    }
    if (!cur.empty() || tk[i].size() != tk[0].size()) return false;
  }
  std::vector<uint8_t> host;
  auto add_phase = [&](const std::vector<const fcgle::GroupRec*>& rs) {
    // one launch per kernel type among rs, in first-appearance order
    std::vector<void (*)(const void*, int, long long, cudaStream_t)> kinds;
    for (auto* r : rs)
      if (std::find(kinds.begin(), kinds.end(), r->launch) == kinds.end()) kinds.push_back(r->launch);
    for (auto fn : kinds) {
      fcgle_batch_ctx::Phase ph{fn, (host.size() + 255) / 256 * 256, 0, 0, {}, {}};
      host.resize(ph.offset);
      for (auto* r : rs) {
        if (r->launch != fn) continue;
        const size_t at = host.size();
        host.insert(host.end(), r->desc.begin(), r->desc.end());
        std::memcpy(host.data() + at + r->ubegin_off, &ph.units, sizeof(long long));
        ph.units += r->units;
        ++ph.n;
        ph.alts = r->alts;
        ph.alt_names = r->alt_names;
      }
      plan.phases.push_back(ph);
    }
  };
  const size_t nt = tk[0].size();
  for (size_t t = 0; t < nt; ++t) {
    size_t inner = 0;
    for (int i = 0; i < ni; ++i) inner = std::max(inner, tk[i][t].size() - 1);
    for (size_t k = 0; k < inner; ++k) {
      std::vector<const fcgle::GroupRec*> rs;
      for (int i = 0; i < ni; ++i)
        if (k + 1 < tk[i][t].size()) rs.push_back(tk[i][t][k]);
      add_phase(rs);
    }
    std::vector<const fcgle::GroupRec*> last;
    for (int i = 0; i < ni; ++i) last.push_back(tk[i][t].back());
    add_phase(last);
  }
  FCGLE_CUDA(cudaMalloc(&plan.dev, std::max<size_t>(host.size(), 256)));
  FCGLE_CUDA(cudaMemcpyAsync(plan.dev, host.data(), host.size(), cudaMemcpyHostToDevice, st));
  FCGLE_CUDA(cudaStreamSynchronize(st));
  tune_plan(plan, st);
  return true;
}

// Per-phase autotuning of a grouped plan: a phase whose kernel has equivalent
// configurations (the plain mode product's ring depths) is timed in each, on
// the batch's own buffers, and the fastest is kept (another configuration
// replaces the recorded one only when 2 % faster).  Plain phases read the
// step's input and write only the scratch tensors of their Tucker operator, so
// running them out of order before the step changes no state.  Synchronous;
// the choices are added to the autotuner's report.
static void tune_plan(fcgle_batch_ctx::Plan& plan, cudaStream_t st) {
  cudaEvent_t e0, e1;
  FCGLE_CUDA(cudaEventCreate(&e0));
  FCGLE_CUDA(cudaEventCreate(&e1));
  int k = 0;
  try {
    for (auto& ph : plan.phases) {
      ++k;
      if (ph.alts.empty()) continue;
      const void* d = static_cast<const uint8_t*>(plan.dev) + ph.offset;
      std::vector<void (*)(const void*, int, long long, cudaStream_t)> cands = {ph.launch};
      cands.insert(cands.end(), ph.alts.begin(), ph.alts.end());
      std::vector<float> us(cands.size(), 0.f);
      for (size_t c = 0; c < cands.size(); ++c) {
        cands[c](d, ph.n, ph.units, st);   // warm-up
        FCGLE_CUDA(cudaEventRecord(e0, st));
        for (int r = 0; r < 3; ++r) cands[c](d, ph.n, ph.units, st);
        FCGLE_CUDA(cudaEventRecord(e1, st));
        FCGLE_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        FCGLE_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        us[c] = 1e3f * ms / 3;
      }
      size_t best = 0;
      for (size_t c = 1; c < cands.size(); ++c)
        if (us[c] < 0.98f * us[0] && us[c] < us[best]) best = c;
      char line[320];
      int n = std::snprintf(line, sizeof(line), "batch phase %d (%d instances, %lld units): X4M2 %.1fus", k, ph.n,
                            ph.units, us[0]);
      for (size_t c = 1; c < cands.size() && n > 0 && n < (int)sizeof(line); ++c)
        n += std::snprintf(line + n, sizeof(line) - n, " %s %.1fus", ph.alt_names[c - 1].c_str(), us[c]);
      if (n > 0 && n < (int)sizeof(line))
        std::snprintf(line + n, sizeof(line) - n, " -> %s", best == 0 ? "X4M2" : ph.alt_names[best - 1].c_str());
      add_tune_report_line(line);
      ph.launch = cands[best];
    }
  } catch (...) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    throw;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
}

fcgle_status fcgle_batch_integrate(fcgle_batch b, int scheme, double tau, int nsteps, double t0,
                                   const void* const* u0, void* const* uT, int use_graph) {
  return guarded([&] {
    if (!b || !u0 || !uT) throw InvalidArg("NULL argument");
    check_scheme(scheme);
    check_tau(tau);
    if (nsteps < 0) throw InvalidArg("nsteps must be >= 0");
    const int n = (int)b->inst.size(), ns = (int)b->streams.size();
    for (int i = 0; i < n; ++i)
      if (!u0[i] || !uT[i]) throw InvalidArg("tensor pointer is NULL");
    // captured steps hold the coefficients and sources they were built with
    unsigned long long gen = 0;
    for (auto* h : b->inst) gen += h->gen;
    if (gen != b->gen_built) {
      batch_drop_cache(b);
      b->gen_built = gen;
    }
    // the caller's stream may be the legacy default stream, which cannot be
    // captured: all work is ordered through the internal origin stream
    auto fork = [&] {
      FCGLE_CUDA(cudaEventRecord(b->fork, b->origin));
      for (auto st : b->streams) FCGLE_CUDA(cudaStreamWaitEvent(st, b->fork, 0));
    };
    auto join = [&] {
      for (int k = 0; k < ns; ++k) {
        FCGLE_CUDA(cudaEventRecord(b->join[k], b->streams[k]));
        FCGLE_CUDA(cudaStreamWaitEvent(b->origin, b->join[k], 0));
      }
    };
    FCGLE_CUDA(cudaEventRecord(b->enter, b->main));
    FCGLE_CUDA(cudaStreamWaitEvent(b->origin, b->enter, 0));
    fork();
    for (int i = 0; i < n; ++i) b->inst[i]->eng->begin_steps(scheme, tau, t0, u0[i]);
    bool replay = use_graph != 0 && nsteps > 0;
    for (int i = 0; i < n && replay; ++i) replay = !b->inst[i]->eng->time_dependent();
    int first = 0;
    if (replay && scheme == FCGLE_LBDF2) {   // step 0 (linearly-implicit Euler) differs from the rest
      for (int i = 0; i < n; ++i) b->inst[i]->eng->one_step(0);
      first = 1;
    }
    bool grouped_done = false;
    if (use_graph == 2 && replay && first < nsteps) {
      join();
      uint64_t tb;
      std::memcpy(&tb, &tau, 8);
      const auto key = std::make_pair(scheme, tb);
      auto it = b->plans.find(key);
      if (it == b->plans.end()) {
        fcgle_batch_ctx::Plan plan;
        bool built = false;
        try {
          built = build_plan(b, first, b->origin, plan);
          if (built) {
            cudaGraph_t g = nullptr;
            FCGLE_CUDA(cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal));
            try {
              for (const auto& ph : plan.phases)
                ph.launch(static_cast<const uint8_t*>(plan.dev) + ph.offset, ph.n, ph.units, b->origin);
            } catch (...) {
              cudaStreamEndCapture(b->origin, &g);
              if (g) cudaGraphDestroy(g);
              throw;
            }
            FCGLE_CUDA(cudaStreamEndCapture(b->origin, &g));
            cudaError_t e = cudaGraphInstantiate(&plan.graph, g, 0);
            cudaGraphDestroy(g);
            FCGLE_CUDA(e);
          }
        } catch (...) {
          if (plan.dev) cudaFree(plan.dev);
          throw;
        }
        if (built) it = b->plans.emplace(key, plan).first;
      }
      if (it != b->plans.end()) {
        for (int k = first; k < nsteps; ++k) {
          FCGLE_CUDA(cudaGraphLaunch(it->second.graph, b->origin));
          ++b->graph_launches;
          b->grouped_kernels += (long long)it->second.phases.size();
        }
        grouped_done = true;
      }
      fork();
    }
    if (grouped_done) {
    } else if (replay && first < nsteps) {
      join();
      uint64_t tb;
      std::memcpy(&tb, &tau, 8);
      auto key = std::make_pair(scheme, tb);
      auto it = b->graphs.find(key);
      if (it == b->graphs.end()) {
        cudaGraph_t g = nullptr;
        FCGLE_CUDA(cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal));
        try {
          fork();
          for (int i = 0; i < n; ++i) b->inst[i]->eng->one_step(first);
          join();
        } catch (...) {
          cudaStreamEndCapture(b->origin, &g);
          if (g) cudaGraphDestroy(g);
          throw;
        }
        FCGLE_CUDA(cudaStreamEndCapture(b->origin, &g));
        cudaGraphExec_t ex = nullptr;
        cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        FCGLE_CUDA(e);
        it = b->graphs.emplace(key, ex).first;
      }
      for (int k = first; k < nsteps; ++k) {
        FCGLE_CUDA(cudaGraphLaunch(it->second, b->origin));
        ++b->graph_launches;
      }
      fork();
    } else {
      for (int k = first; k < nsteps; ++k)
        for (int i = 0; i < n; ++i) b->inst[i]->eng->one_step(k);
    }
    for (int i = 0; i < n; ++i) b->inst[i]->eng->end_steps(uT[i]);
    join();
    FCGLE_CUDA(cudaEventRecord(b->leave, b->origin));
    FCGLE_CUDA(cudaStreamWaitEvent(b->main, b->leave, 0));
  });
}

fcgle_status fcgle_batch_launch_count(fcgle_batch b, long long* kernels, long long* graph_launches) {
  return guarded([&] {
    if (!b) throw InvalidArg("NULL batch");
    long long k = 0;
    for (auto* h : b->inst) k += h->eng->launches;
    k += b->grouped_kernels;
    if (kernels) *kernels = k;
    if (graph_launches) *graph_launches = b->graph_launches;
  });
}

fcgle_status fcgle_batch_destroy(fcgle_batch b) {
  return guarded([&] { batch_free(b); });
}

fcgle_status fcgle_autotune_report(char* buf, size_t size, size_t* needed) {
  return guarded([&] {
    const std::string r = plain_tune_report();
    if (needed) *needed = r.size() + 1;
    if (buf && size > 0) {
      const size_t n = std::min(size - 1, r.size());
      std::memcpy(buf, r.data(), n);
      buf[n] = 0;
    }
  });
}

const char* fcgle_status_string(fcgle_status s) {
  switch (s) {
    case FCGLE_OK: return "FCGLE_OK";
    case FCGLE_ERR_INVALID_ARG: return "FCGLE_ERR_INVALID_ARG";
    case FCGLE_ERR_NOMEM: return "FCGLE_ERR_NOMEM";
    case FCGLE_ERR_CUDA: return "FCGLE_ERR_CUDA";
    case FCGLE_ERR_NUMERIC: return "FCGLE_ERR_NUMERIC";
    case FCGLE_ERR_TIMEOUT: return "FCGLE_ERR_TIMEOUT";
    case FCGLE_ERR_UNSUPPORTED: return "FCGLE_ERR_UNSUPPORTED";
  }
  return "FCGLE_ERR_UNKNOWN";
}

const char* fcgle_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
