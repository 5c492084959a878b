// Internal declarations shared by the libusbs translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "usbs.h"

// Read-only qualifiers of the kernel bodies.  A kernel that writes a buffer and reads it
// again later in the same launch (the batched solver runs a whole solve in one launch)
// must not read it through the non-coherent read-only path, so that translation unit
// defines USBS_PLAIN_LOADS before including this header.
#ifdef USBS_PLAIN_LOADS
#define USBS_RESTRICT
#define USBS_LDG(p) (*(p))
#else
#define USBS_RESTRICT __restrict__
#define USBS_LDG(p) __ldg(p)
#endif

namespace usbs {

constexpr int KB = 8;            // Lanczos block width and max k_c (V is n x 8, zero-padded)
constexpr int KSV = 36;          // svec dimension for an 8 x 8 matrix
constexpr int JMAX = 64;         // max Lanczos basis columns (8 blocks of 8)
constexpr int NBMAX = JMAX / KB + 1;  // basis blocks incl. the residual block
constexpr int RMAX = 32;         // max sketch rank
constexpr int AUG = 40;          // augmented Gram width: 36 svec + ax + w + 2 pad
constexpr int RED_GRID_MAX = 4 * 152;   // most CTAs of any reducing kernel
constexpr int THREADS = 256;

// ---- device-resident FP64 scalars of one instance ------------------------------------
struct DevScalars {
  // iterate state (scaled units)
  double f_y;          // f(y_t)
  double cx;           // <C, Xbar_t>
  double tr;           // tr Xbar_t
  // result of the subproblem of the current step
  double eta_hat, eta;
  double S_hat[64];    // 8 x 8 row-major (k_c x k_c used)
  double S[64];
  double theta_ipm[4]; // zeta, omega, mu, unused
  double cx_new, tr_new;
  // candidate and model value
  double bty, axy;     // <b, y~>, <A Xbar, y~>
  double f_cand, f_hat, lam_max;
  double relgap, relinf, relinf_max;
  double dnu;          // ||nu_new - nu_old|| of the last alternation pass
  double Vc[64];       // V^T C V
  double B_sketch[KB * RMAX];  // V^T Psi (k x r)
  int descent, ipm_iters, has_eta, status;
  int t, n_alt, matvecs, pad;
  // certification of f(y) at the centre (usbs_solve with certify_restarts > 0)
  double f_cert, lam_cert;
  // the primal iterate X_{t+1} = eta Xbar_t + V S V^T (gates, objective); cx and tr above
  // hold Xbar's, which differ from these when k_p > 0
  double cx_it, tr_it;
  double cx_prev, tr_prev;   // Xbar_t's <C, Xbar>, tr Xbar before the step's update
  // past information (k_p > 0): S = S_p + S_c and the k_p leading eigenvectors Q_p of S
  double Sp[64], Sc[64], Qp[64];
  // the model value by the App. B.1 IPM (model_value_ipm = 1) beside the closed form
  double f_hat_ipm, f_hat_closed;
  int ipm_iters_b1, pad2;
};

// ---- Lanczos device state -------------------------------------------------------------
struct DevLanczos {
  double T[JMAX * JMAX];       // projected matrix Q^T M Q, row-major J x J
  double Y[JMAX * JMAX];       // Ritz vectors (columns), row-major J x J
  double theta[JMAX];          // Ritz values, descending
  double R[64];                // R factor of the last orthonormalised block (8 x 8, upper)
  double Rinv[64];             // its inverse
  double Rlast[64];            // R of the residual block of the cycle
  double res[KB];              // residual norms of the top k_c Ritz pairs
  double normest;              // running estimate of |M|
  int dcol[8];                 // per column of the current block: 1 = replace by a random
                               // vector, 2 = zero it (still dependent after two passes)
  int defl;                    // mask of the second pass: the first pass replaced a column
  int defl2;                   // mask of the third pass: the second pass replaced a column
  int converged;
  int cycles;
  int status;                  // USBS_ENUMERIC if the projected matrix went non-finite
  int sweeps;                  // Jacobi sweeps summed over the cycles of this solve
  int defl_seen;               // a first pass of this cycle found a deficient column
  int redo;                    // the cycle ran without its masked passes but needed them:
                               // its Rayleigh-Ritz step was skipped, the host reruns it
};

// TMA tensor map of one n x 8 FP32 buffer of a context (tc_orth.cu)
struct TmaEntry {
  const char* base;
  size_t bytes;
  CUtensorMap map;
};

template <typename T>
struct Buf {
  T* p = nullptr;
  size_t n = 0;
};

struct Ctx {
  // sizes and parameters
  int64_t n = 0, m = 0, nnzA = 0;
  int nnz_off = 0;              // off-diagonal entries of the merged operator pattern
  usbs_params prm{};
  int kc = 8, r = 0, J = 64, keep = 32;
  int kp = 0;                   // past-information columns (Sec. 3); V holds kdim = kc + kp
  int kdim = 8;
  int kconv = 8;                // top Ritz pairs whose residuals end an eigen solve
  bool fp64 = false;
  bool has_offdiag_A = false;
  bool any_ineq = false;
  double c_scale = 1.0, tau = 1.0, bnorm = 0.0, alpha = 2.0;
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int num_sms = 152;
  std::string err;
  bool started = false;         // an iterate exists (cold start done)
  bool debug = false;           // USBS_DEBUG=1: per-block-step checks on the host
  bool speculate = true;        // run Lanczos cycles without the masked passes, rerun a cycle
                                // that needed them (USBS_NO_SPECULATE=1 turns this off)
  long long total_matvecs = 0;
  bool use_tc = false;          // FP32 Gram-Schmidt and restart tiles on tcgen05 (USBS_TCGEN05=1)
  std::vector<TmaEntry> tma;    // tensor maps of the FP32 n x 8 buffers

  // operator (scaled): merged off-diagonal CSR pattern + diagonal
  int* rowptr = nullptr;        // n+1
  int* col = nullptr;           // nnz_off
  double* valC64 = nullptr;     // base C values (scaled), FP64
  void* valM = nullptr;         // effective values of C - A*(y), T
  void* valC = nullptr;         // base values in T (for C V)
  double* diagC64 = nullptr;    // n
  void* dM = nullptr;           // diag of C - A*(y), T
  void* dC = nullptr;           // diag of C, T
  // A*(y) scatter lists (FP64): diagonal and off-diagonal slots
  int* diag_ptr = nullptr; int* diag_con = nullptr; double* diag_val = nullptr;
  int* slot_ptr = nullptr; int* slot_con = nullptr; double* slot_val = nullptr;
  // constraints in constraint-major order
  int* con_ptr = nullptr;       // m+1
  int* ent_i = nullptr; int* ent_j = nullptr;
  void* ent_v = nullptr;        // T
  double* b = nullptr;          // scaled b
  uint8_t* ineq = nullptr;

  // iterate (FP64 m-vectors)
  double* y = nullptr;          // y_t
  double* ycand = nullptr;      // y~_{t+1}
  double* ax = nullptr;         // A Xbar_t
  double* axnew = nullptr;      // A X_{t+1}
  double* nu = nullptr;
  double* ytmp = nullptr;       // operator argument for usbs_extreme_eigs
  // n-sized (T)
  void* V = nullptr;            // n x 8
  void* Vnew = nullptr;         // n x 8
  void* W = nullptr;            // n x 8
  void* Q = nullptr;            // basis, NBMAX blocks of n x 8
  void* Q2 = nullptr;           // restart target
  float* P = nullptr;           // n x r
  float* Psi = nullptr;         // n x r
  // scalars, Lanczos state, reductions
  DevScalars* sc = nullptr;
  DevLanczos* lz = nullptr;
  double* partials = nullptr;   // max_parts x PART_STRIDE
  int max_parts = 1;            // rows of partials: the largest grid of a reducing kernel
  double* red = nullptr;        // reduced outputs (several regions)
  DevScalars* h_sc = nullptr;   // pinned host mirror
  DevLanczos* h_lz = nullptr;
  uint64_t seed = 0;
  uint64_t rng_counter = 1;
  int64_t spec_redos = 0;       // speculative Lanczos cycles that had to run again
  // measurement
  long long launches = 0;
  bool prof = false;
  double prof_ms[USBS_NUM_KINDS] = {};
  long long prof_n[USBS_NUM_KINDS] = {};
  double prof_bytes[USBS_NUM_KINDS] = {};
  struct PendingEv { cudaEvent_t a, b; int kind; };
  std::vector<PendingEv> prof_pending;
  std::vector<cudaEvent_t> ev_pool;
  // outcome of the last batched solve of this context (batch.cu)
  int batch_iters = 0, batch_converged = 0, batch_descent = 0, batch_status = 0;
  int batch_last_matvecs = 0, batch_n_alt = 0;
  long long batch_matvecs = 0;
};

// ---- batched solver (batch.cu) -------------------------------------------------------------
// A context the persistent batched kernel can solve (its basis size is instantiated and
// no per-step host work is enabled).
bool batch_eligible(const Ctx* c);
// Size bucket of an instance for the batched solver (n < 256, 512, 1024, 2048, larger).
int batch_bucket(int64_t n);
// Cold-start solves of all contexts (same precision, basis and size bucket) in one launch of
// the persistent kernel (a CUDA graph replayed per bucket) on stream st.
int batch_run(const std::vector<Ctx*>& cs, cudaStream_t st, double tol, std::string& err);
// usbs_result of a context's last batched solve, as usbs_solve would report it.
int batch_result(Ctx* c, usbs_result* out);

void prof_resolve(Ctx* c);

// Brackets one kernel launch: counts it and, with profiling on, records events.
struct LaunchScope {
  Ctx* c;
  int kind;
  cudaEvent_t a = nullptr;
  LaunchScope(Ctx* c_, int kind_, double bytes = 0.0) : c(c_), kind(kind_) {
    c->launches++;
    if (c->prof) {
      c->prof_bytes[kind] += bytes;
      a = take_event();
      cudaEventRecord(a, c->stream);
    }
  }
  ~LaunchScope() {
    if (c->prof && a) {
      cudaEvent_t b = take_event();
      cudaEventRecord(b, c->stream);
      c->prof_pending.push_back({a, b, kind});
      if (c->prof_pending.size() > 8192) prof_resolve(c);
    }
  }
  cudaEvent_t take_event() {
    if (!c->ev_pool.empty()) {
      cudaEvent_t e = c->ev_pool.back();
      c->ev_pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
};
#define USBS_LAUNCH(c, kind) LaunchScope usbs_launch_scope_(c, kind)
// same, adding the launch's algorithmic bytes (each input read once, each output
// written once) to the kind's total
#define USBS_LAUNCH_B(c, kind, bytes) LaunchScope usbs_launch_scope_(c, kind, (double)(bytes))

// regions inside Ctx::red (doubles)
constexpr int RED_H = 0;          // 8 blocks x 64
constexpr int RED_H2 = 512;       // 8 blocks x 64
constexpr int RED_GRAM = 1024;    // 64
constexpr int RED_AUG = 1152;     // AUG x AUG (full)
constexpr int RED_VEC = 2816;     // 36 + scalars (alternation / candidate)
constexpr int RED_SK = 2944;      // 8 x 32 sketch B
constexpr int RED_VC = 3200;      // 64, V^T C V
constexpr int RED_CERT = 3328;    // 8: <b, y> of the certification
constexpr int RED_TOTAL = 3336;
constexpr int PART_STRIDE = 1024; // doubles per CTA in partials

// ---- error helpers ---------------------------------------------------------------------
#define USBS_CUDA_TRY(ctx, call)                                                   \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      (ctx)->err = std::string(#call) + ": " + cudaGetErrorString(e_);             \
      return USBS_ECUDA;                                                           \
    }                                                                              \
  } while (0)

#define USBS_TRY(expr)                                                             \
  do {                                                                             \
    int rc_ = (expr);                                                              \
    if (rc_ != USBS_OK) return rc_;                                                \
  } while (0)

int check_launch(Ctx* c, const char* what);

// ---- launchers (bulk.cu) -----------------------------------------------------------------
template <typename T> struct Bulk {
  static void setup_operator(Ctx* c, const double* y);
  static void spmm(Ctx* c, const void* valM, const void* dM, const void* X, void* Y);
  static void gstats(Ctx* c, const void* V, const double* ax, const double* y, int nparts);
  static void alt_pass(Ctx* c, const void* V, int nparts);
  static void xupdate(Ctx* c, const void* V, int nparts);
  static void vt_psi(Ctx* c, const void* V, int nparts);
  static void sketch_update(Ctx* c, const void* V, const double* S, const double* Bsk, float* P,
                            const float* Psi, const double* eta_dev, double eta_host);
  static void constraint_eval(Ctx* c, const void* V, const double* S, double* z);
  // out = eta ax + A(V S V^T), eta on the device (Xbar's constraint values when k_p > 0)
  static void constraint_axpy(Ctx* c, const void* V, const double* S, const double* eta_dev,
                              const double* ax, double* out);
  // W = [V Q_p | U_{:, :k_c} | 0] (the block whose QR is V_{t+1} when k_p > 0)
  static void vnext(Ctx* c, const void* V, const double* Qp, const void* U, void* W);
};

// shared-memory-staged block Gram-Schmidt kernels (orth.cu); grid = orth_grid(c, n)
template <typename T> struct Orth {
  // proj, update and gram_xy return the grid they launched (the partials to reduce)
  static int proj(Ctx* c, const void* Qb, int nb, const void* W, const int* mask);
  static int update(Ctx* c, const void* Qb, int nb, void* W, const int* mask);
  static void finalize(Ctx* c, const void* Qb, int nb, const void* W, void* out, const int* mask,
                       uint64_t seed);
  static void restart(Ctx* c, const void* Qb, int J, int nout, const double* Y, void* out,
                      const void* resid, int resid_slot);
  // X^T Y of two n x 8 blocks (partials in the layout of proj with one block)
  static int gram_xy(Ctx* c, const void* X, const void* Y);
};
// CTAs of a tiled Gram-Schmidt launch: one per tile of rows, at most what stays resident
// on every SM at once for that kernel and shared-memory size, at most max_parts
int orth_grid(Ctx* c, int64_t rows, const void* kernel, size_t smem);
// tcgen05 tiles of the mixed-precision path (tc_orth.cu).  tc_proj / tc_update return the
// grid they launched (0: no tensor map for a buffer, nothing launched); tc_final /
// tc_restart return whether they launched.
void tc_register(Ctx* c);
int tc_proj(Ctx* c, const void* Q, int nb, const void* W, const int* mask);
int tc_update(Ctx* c, const void* Q, int nb, void* W, const int* mask);
bool tc_final(Ctx* c, const void* Q, int nb, const void* W, void* out, const int* mask, uint64_t seed);
bool tc_restart(Ctx* c, const void* Q, int J, int nout, const double* Y, void* out, const void* resid,
                int resid_slot);
// rows of partials a context needs: ceil(max(n, m) / 64) + 1, at most RED_GRID_MAX
int64_t parts_needed(int64_t n, int64_t m);

int red_grid(Ctx* c, int64_t rows, int rows_per_cta);
void reduce_partials(Ctx* c, int nparts, int nvals, double* out, const int* mask = nullptr);

void reduce_max_slot(Ctx* c, int nparts, int slot, double* out);

// ---- small single-CTA kernels (small.cu) -------------------------------------------------
void launch_chol_block(Ctx* c, int j, int nb, int write_T, int is_resid, int defl_pass);
void launch_ritz(Ctx* c, int J, int keep, int spec);
void launch_ipm(Ctx* c, int first_pass);
// App. B.1: the model value at y~ by the IPM (model_value_ipm = 1), after k_xupdate's sums
void launch_ipm_b1(Ctx* c);
void launch_finish(Ctx* c);
void launch_commit(Ctx* c);
void launch_cold(Ctx* c);
void launch_begin_step(Ctx* c);
void launch_lanczos_reset(Ctx* c);
// f(y) at the centre from the certifying eigen solve's top Ritz value and <b, y> (in
// red + RED_CERT); keeps the larger value of f(y) and re-evaluates the gap
void launch_certify(Ctx* c);
// S = S_p + S_c split of the k_p largest eigenpairs and Xbar's scalars (k_p > 0)
void launch_kp_split(Ctx* c);
// out = <a, b> over m FP64 entries (per-CTA partials reduced in a fixed order)
void launch_dot(Ctx* c, const double* a, const double* b, int64_t m, double* out);

// device address of a member of a device-resident struct (no dereference on the host)
#define DEV_FIELD(base, Type, field, Elem) \
  reinterpret_cast<Elem*>(reinterpret_cast<char*>(base) + offsetof(Type, field))

}  // namespace usbs
