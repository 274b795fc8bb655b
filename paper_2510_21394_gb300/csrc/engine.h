// Host-side engine of one FCGLE handle: spectral setup, buffers and the
// time-stepping schemes, all enqueued on the handle's stream.
#pragma once

#include <map>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/fcgle.h"
#include "common.h"

namespace fcgle {

struct InvalidArg : std::runtime_error {
  using std::runtime_error::runtime_error;
};
struct Unsupported : std::runtime_error {
  using std::runtime_error::runtime_error;
};
struct NumericError : std::runtime_error {
  using std::runtime_error::runtime_error;
};
struct DeviceTimeout : std::runtime_error {
  using std::runtime_error::runtime_error;
};

// Per-direction FP64 spectral data, computed once at setup on the host.
struct Direction {
  int n = 0, p = 0;
  double h = 0;
  std::vector<double> Q;     // n x n row-major, column j = eigenvector j
  std::vector<double> lam;   // n eigenvalues of D_mu (negative)
};

class EngineBase {
 public:
  virtual ~EngineBase() = default;
  virtual void set_stream(cudaStream_t st) = 0;
  virtual void set_source(int nterms, const double* sig, const void* const* S_user) = 0;
  // new nu, eta, gamma, kappa, zeta (the eigendecompositions do not depend on them)
  virtual void set_coefficients(double nu, double eta, double gamma, double kappa, double zeta) = 0;
  // how e^{theta K} is applied (fcgle_exp_form); FP64 engines always use the
  // Kronecker-product form and only validate the value
  virtual void set_exp_form(int form) {
    if (form != FCGLE_EXP_TUCKER && form != FCGLE_EXP_KRON) throw InvalidArg("unknown exponential form");
  }
  // how a Tucker operator of a 3D split-BF16 handle is run (fcgle_tucker_form);
  // other engines only validate the value
  virtual void set_tucker_form(int form) {
    if (form < FCGLE_TUCKER_AUTO || form > FCGLE_TUCKER_SLAB) throw InvalidArg("unknown Tucker-operator form");
    if (form == FCGLE_TUCKER_SLAB) throw Unsupported("the slab-fused form is a 3D split-BF16 form");
  }
  virtual void apply_f(int func, int k, double theta, const void* v, void* out) = 0;
  virtual void step(int scheme, double tau, double t, void* u) = 0;
  virtual void integrate(int scheme, double tau, int nsteps, double t0, const void* u0, void* uT) = 0;
  virtual void integrate_host(int scheme, double tau, int nsteps, double t0, const void* u0, void* uT) = 0;
  virtual double norm(const void* u) = 0;
  // discrete adjoint of Lawson-RK2 (adjoint.h); user-layout device tensors, synchronous
  virtual void adjoint(int scheme, double tau, int nsteps, double t0, const void* u0, const void* target,
                       int ckpt_every, void* grad_u0, double* grad_params, double* loss) = 0;
  virtual void mode_product(int mu, bool fwd, const void* X, void* Y) = 0;
  // flags: bit 0 forward (Q^T), bit 1 split-bf16 input and output, bit 2 the
  // precise (split-TF32) product on FP32 input and output, bit 3 the
  // slab-fused modes 1 + 2, bit 4 the natural-order last product (bits 1-4:
  // BF16X3 only)
  virtual void mode_product_flags(int mu, int flags, const void* X, void* Y) {
    if (flags & 30) throw InvalidArg("flags bits 1 to 4 need a BF16X3 handle");
    mode_product(mu, flags & 1, X, Y);
  }
  virtual size_t internal_elems() const = 0;
  // f(theta lam) for lam = (nu + i eta) s_j, host lists, evaluated on the device
  // by the arithmetic the handle's kernels use; synchronous
  virtual void spectral_scalars(int func, int k, double theta, int count, const double* s_host, double* out_host,
                                int flags) = 0;
  // stepping interface (batched CUDA graphs): pack u0 and build the loop's entry
  // state; enqueue step n; unpack the state.  No host synchronisation inside
  // one_step, so a step can be captured into a graph.
  virtual void begin_steps(int scheme, double tau, double t0, const void* u0) = 0;
  virtual void one_step(int n) = 0;
  virtual void end_steps(void* uT) = 0;
  // true if the step depends on t through the source (a captured step then
  // cannot be replayed for other n)
  virtual bool time_dependent() const = 0;
  virtual size_t elem_bytes() const = 0;
  virtual int device_error() = 0;   // reads and clears the device error flag (synchronises)
  // times the kernel configurations this handle can choose between and records
  // the fastest (process-wide, per problem shape); synchronous; no-op by default
  virtual void autotune() {}
  // Grouped batch launches: while a recorder is set, every mode product of
  // one_step is recorded (as a kernel descriptor) instead of launched.
  // Returns false if the engine has no grouped form (FP64, d == 1).
  virtual bool set_recorder(std::vector<struct GroupRec>* rec) { return rec == nullptr; }
  long long launches = 0;
};

// One recorded mode product: the descriptor of one problem of a grouped
// persistent launch, and the launcher of that kernel type.  Records with the
// same launcher can share a launch (their descriptors concatenated).
struct GroupRec {
  bool last;   // last mode product of a Tucker operator (carries the scheme's epilogue)
  void (*launch)(const void* descs, int n, long long units, cudaStream_t st);
  // launchers of equivalent kernel configurations that read the same descriptor
  // format (the autotuner of a batch times them per phase); may be empty
  std::vector<void (*)(const void*, int, long long, cudaStream_t)> alts;
  std::vector<std::string> alt_names;
  size_t ubegin_off;          // byte offset of the descriptor's first-unit field
  std::vector<uint8_t> desc;  // the descriptor bytes (size = stride in the array)
  long long units;
};

// D_mu of direction mu (Eq. Dnalpha / Eq. FD4) and its FP64 eigendecomposition
// (Eq. diag), residual-checked.
Direction spectral_direction(const fcgle_params& prm, int mu);

std::unique_ptr<EngineBase> make_engine(const fcgle_params& prm, cudaStream_t st);
// the plain-product autotuner's timings and choices so far, one line per shape
// (and one per tuned phase of a batch)
std::string plain_tune_report();
void add_tune_report_line(const std::string& line);
std::unique_ptr<EngineBase> make_engine_b3(const fcgle_params& prm, cudaStream_t st);

}  // namespace fcgle
