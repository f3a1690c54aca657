// fde_host.cu -- context, plane-wave bases, plans and the C ABI of include/fde.h.
//
// Host code orchestrates the device work of one GPU: it builds the plane-wave spheres and
// their FFT column maps, the twiddle tables, the projector tables and the work buffers,
// and runs the block-Davidson eigensolver, the subsystem SCF and the freeze-and-thaw
// cycle, whose every grid-, band- and subspace-sized step is a kernel of this library.
// Only scalars (eigenvalues, norms, energies, DIIS coefficients) travel to the host.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <memory>
#include <string>
#include <vector>

#include "fde.h"
#include "grid_kernels.h"
#include "hostmath.h"
#include "kernels.h"
#include "prof.h"
#include "precond.h"
#include "small.h"

namespace fde {

thread_local Profiler* tl_prof = nullptr;

struct Err {
  fde_status st;
  std::string msg;
};

#define CK(x)                                                                                   \
  do {                                                                                          \
    cudaError_t e_ = (x);                                                                       \
    if (e_ != cudaSuccess) throw Err{FDE_ECUDA, std::string(#x) + ": " + cudaGetErrorString(e_)}; \
  } while (0)
#define REQ(c, s, m)              \
  do {                            \
    if (!(c)) throw Err{(s), (m)}; \
  } while (0)

// Every device (re)allocation or release bumps this counter; a captured CUDA graph whose
// counter value is stale may reference freed buffers and is captured again.
static unsigned long long g_alloc_generation = 0;

// FDE_TRACE=1 in the environment prints one line per SCF iteration to stderr.
static int trace_level() {
  static int lv = -1;
  if (lv < 0) {
    const char* e = getenv("FDE_TRACE");
    lv = e ? atoi(e) : 0;
  }
  return lv;
}

template <typename X> struct DBuf {
  X* p = nullptr;
  size_t n = 0;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
  DBuf& operator=(DBuf&& o) noexcept {
    if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
    return *this;
  }
  ~DBuf() { release(); }
  void release() {
    if (p) {
      cudaFree(p);
      ++g_alloc_generation;
    }
    p = nullptr;
    n = 0;
  }
  void alloc(size_t count) {
    release();
    ++g_alloc_generation;
    if (count) {
      cudaError_t e = cudaMalloc(&p, count * sizeof(X));
      if (e != cudaSuccess) { p = nullptr; throw Err{FDE_ENOMEM, "cudaMalloc failed"}; }
      n = count;
    }
  }
  void ensure(size_t count) {
    if (count > n) alloc(count);
  }
};

static const long double kPiL = 3.141592653589793238462643383279502884L;

template <typename T> struct Plans {
  DBuf<cplx<T>> tw[3];
  FftPlans<T> fp;
};

static void factorize(int n, int* radix, int* nst) {
  int m = n, k = 0;
  while (m % 4 == 0 && k < kMaxStages) { radix[k++] = 4; m /= 4; }
  while (m % 2 == 0 && k < kMaxStages) { radix[k++] = 2; m /= 2; }
  while (m % 3 == 0 && k < kMaxStages) { radix[k++] = 3; m /= 3; }
  while (m % 5 == 0 && k < kMaxStages) { radix[k++] = 5; m /= 5; }
  REQ(m == 1, FDE_EUNSUPPORTED, "grid sizes must factor into 2, 3 and 5");
  *nst = k;
}

template <typename T> static void make_plans(Plans<T>& P, const int grid[3], cudaStream_t) {
  LinePlan<T>* lp[3] = {&P.fp.p1, &P.fp.p2, &P.fp.p3};
  for (int a = 0; a < 3; ++a) {
    const int n = grid[a];
    std::vector<cplx<T>> h(n);
    for (int m = 0; m < n; ++m) {
      const long double ang = 2.0L * kPiL * (long double)m / (long double)n;
      h[m] = mk<T>((T)cosl(ang), (T)(-sinl(ang)));
    }
    P.tw[a].alloc(n);
    CK(cudaMemcpy(P.tw[a].p, h.data(), n * sizeof(cplx<T>), cudaMemcpyHostToDevice));
    lp[a]->n = n;
    factorize(n, lp[a]->radix, &lp[a]->nstages);
    lp[a]->tw = P.tw[a].p;
  }
}

// Host-side physics that is not on the data path (sphere, Ewald, occupations, Pulay
// coefficients) lives in hostmath.cu.

// ---- per-(subsystem, k) and per-subsystem state ---------------------------------------------
template <typename T> struct KP {
  int npw = 0;
  double kfrac[3] = {0, 0, 0}, kc[3] = {0, 0, 0};
  std::vector<int> miller;
  std::vector<double> kin;
  DBuf<int> cols;
  SphereDev sp{};
  DBuf<T> kin_d;
  DBuf<cplx<T>> beta;
  DBuf<cplx<T>> X, HX;
  std::vector<double> eig, occ;
  bool have_orbitals = false;
  bool have_eig = false;
};

template <typename T> struct Sub {
  int natoms = 0, nproj_atom = 0, nproj = 0, nb = 0, nk = 0;
  double rc = 0, nelec = 0, smearing = 0;
  int smear_kind = FDE_SMEAR_FERMI;
  std::vector<double> pos, Z, sigma, D, kpts, wk;
  std::vector<KP<T>> kp;
  KbBlock Dblk{};  // per-atom projector coupling
  DBuf<double> rho, veff;
  DBuf<T> vplane;
  double entropy = 0, mu = 0;
  // ultrasoft-like augmentation (aug_sigma > 0): overlap S = 1 + sum_a |beta_a> q <beta_a|,
  // charges q_ij g_a(r) in the density, and the coupling of each atom screened by its potential
  bool uspp = false;
  double aug_sigma = 0;
  std::vector<double> Q;
  KbBlock Qblk{};
  DBuf<double> aug_pos, Dscr;
};

struct EnergyParts {
  double Eloc = 0, EH = 0, Exc = 0, Ttot = 0, Tsub = 0, Exc_sub = 0, EH_sub = 0;
};

// ---- the engine ------------------------------------------------------------------------------
struct Engine {
  virtual ~Engine() = default;
  virtual int add_subsystem(const fde_subsys_desc* d) = 0;
  virtual void get_basis(int sub, int k, int* npw, int* miller) = 0;
  virtual void set_density(int sub, const double* rho, int on_device) = 0;
  virtual void get_density(int sub, double* d_rho) = 0;
  virtual void build_vemb(double* d_out, fde_energies* e) = 0;
  virtual void set_veff(int sub, const double* d_v) = 0;
  virtual void apply_h(int sub, int k, const void* psi, void* hpsi, int nb) = 0;
  virtual void apply_h_host(int sub, int k, const double* psi, double* hpsi, int nb) = 0;
  virtual void apply_h_all() = 0;
  virtual void apply_s_dev(int sub, int k, const void* psi, void* spsi, int nb) = 0;
  virtual void init_orbitals(int sub, int k, const double* raw) = 0;
  virtual void set_orbitals(int sub, int k, const double* d_psi) = 0;
  virtual void get_orbitals(int sub, int k, double* d_psi, double* eig, double* occ) = 0;
  virtual fde_status subspace_solve(int sub, int k, double tol, int max_iter, int* iters, int precond) = 0;
  virtual void update_density(int sub) = 0;
  virtual void energy(fde_energies* out) = 0;
  virtual fde_status scf_subsystem(int sub, double tol, int max_scf, fde_energies* out) = 0;
  virtual fde_status freeze_thaw(double tol, int max_scf, fde_energies* out, const double* start) = 0;
  virtual fde_status scf_refresh(double tol, int max_scf, fde_energies* out) = 0;
  virtual void set_symmetry(int nops, const int* ops) = 0;
  virtual double delta_rho(const double* d_ref) = 0;
  virtual void sync() = 0;
  virtual void fft3d(void* data, int sign) = 0;
  virtual void fft3d_f64(double2* data, int sign, int arith) = 0;
  virtual void precond_set_weights(const float* h) = 0;
  virtual void precond_get_weights(float* h, float* hb) = 0;
  virtual void precond_harvest(int sub, int k, const double* raw, int n) = 0;
  virtual void precond_add_pairs(int sub, int k, int n, const double* r, const double* d, const double* tb) = 0;
  virtual void precond_clear() = 0;
  virtual void precond_loss_grad(double* grad, double* loss) = 0;
  virtual void precond_train(int steps, double lr, double* l0, double* l1) = 0;
  virtual void precond_apply(int sub, int k, const void* r, void* w, int nb, const double* tband) = 0;
  virtual void set_precond_mode(int mode) = 0;
  virtual void stats(long long* dav, long long* hpsi) = 0;
  virtual void set_precond_record(int n) = 0;
  virtual void hot_step(bool use_graph) = 0;
  virtual void hot_step_host(const double* const* rho, const double* const* psi, double* const* hpsi) = 0;
  virtual void get_hpsi(int sub, int k, double* d_hpsi) = 0;
  virtual int nsub() const = 0;
  virtual long long grid_points() const = 0;
  virtual void shape(int sub, int* nb, int* nk) = 0;
  virtual int npw(int sub, int k) = 0;
  virtual void set_eig_occ(int sub, int k, const double* eig, const double* occ) = 0;
  virtual void set_subsystem_entropy(int sub, double ts) = 0;
  virtual double subsystem_entropy(int sub) = 0;
};

template <typename T> struct EngineT : Engine {
  using C = cplx<T>;
  cudaStream_t st;
  double A[3][3], B[3][3], omega;
  int grid[3];
  GridDims g;
  long long nr;
  CellDev cell;
  double ecut;
  fde_func_desc func;
  Plans<T> plans;
  Plans<double> plans64;
  Plans<dd> plansdd;  // mixed contexts: double-float transforms of the density and its gradients
  std::vector<std::unique_ptr<Sub<T>>> subs;
  bool locked = false;  // no more subsystems once the local potential exists
  DBuf<double> vloc;
  double enn = 0;
  // grid work
  // Work grids of the embedding-potential build.  Its transforms run in FP64 in both
  // precisions: FP32 gradients of the density are noise where the density is small (the
  // vacuum above the slab), and the GGA potentials amplify that noise by rho^{-4/3}.
  DBuf<double2> cb[2];                // packed transform / potential; rho_tot(G)
  std::vector<DBuf<double2>> packs;   // per subsystem pair: packed gradient grids
  DBuf<double2> cvl;
  DBuf<double> rho_tot, vpart, htot[3], partial, scal;
  DBuf<unsigned> status;
  // band work
  DBuf<C> scratch;
  DBuf<double2> gwork, Pm, Qm;
  DBuf<C> V, HV, V2, HV2, R, Pb, HPb;
  DBuf<double2> S, Hs, L, Li, Ht, Y, Cc, tmp, jwork;
  DBuf<double> wv, dnorm, deps, dtb, hwork;
  DBuf<int> didx;
  DBuf<double> rho_plane, occw;
  // Pulay histories (one for the subsystem SCF, one per subsystem for the refreshed SCF)
  // and freeze-and-thaw copies
  struct PulayHist {
    std::vector<DBuf<double>> in, res;
    int len = 0, head = 0;
  };
  PulayHist hist, hist_all;
  DBuf<double> rho_in, frozen, fresh;
  DBuf<const double*> dptrs;
  DBuf<double> dcoef;
  // host staging
  double* pin = nullptr;
  size_t pin_n = 0;

  EngineT(const fde_cell_desc* c, const fde_func_desc* f, cudaStream_t s) : st(s) {
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        A[i][j] = c->lattice[i][j];
        if (i != j) REQ(c->lattice[i][j] == 0.0, FDE_EUNSUPPORTED, "only orthorhombic (diagonal) lattices");
      }
    for (int i = 0; i < 3; ++i) {
      REQ(A[i][i] > 0, FDE_EINVAL, "lattice diagonal must be positive");
      REQ(c->grid[i] >= 2 && c->grid[i] <= kMaxLine, FDE_EUNSUPPORTED, "grid sizes must be in [2, 320]");
      grid[i] = c->grid[i];
    }
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) B[i][j] = (i == j) ? 2.0 * M_PI * (1.0 / A[i][i]) : 0.0;
    omega = A[0][0] * A[1][1] * A[2][2];
    g = GridDims{grid[0], grid[1], grid[2]};
    nr = (long long)grid[0] * grid[1] * grid[2];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) cell.b[i][j] = B[i][j];
    cell.omega = omega;
    ecut = c->ecut_ha;
    REQ(ecut > 0, FDE_EINVAL, "ecut must be positive");
    func = *f;
    REQ(func.xc == FDE_XC_LDA || func.xc == FDE_XC_PBE, FDE_EINVAL, "unknown xc");
    REQ(func.kedf >= 0 && func.kedf <= 2, FDE_EINVAL, "unknown kinetic functional");
    REQ((size_t)g.n1 * (g.n2 + 1) * sizeof(C) <= 227 * 1024, FDE_EUNSUPPORTED,
        "an (x, y) plane must fit in shared memory");
    REQ(g.n1 <= kMaxPlane && g.n2 <= kMaxPlane, FDE_EUNSUPPORTED, "n1 and n2 must be at most 160");
    make_plans(plans, grid, st);
    make_plans(plans64, grid, st);
    if constexpr (sizeof(T) == 4) make_plans(plansdd, grid, st);
    for (auto& b : cb) b.alloc(nr);
    rho_tot.alloc(nr);
    vpart.alloc(nr);
    for (auto& b : htot) b.alloc(nr);
    partial.alloc(64 * (size_t)grid_red_blocks());
    scal.alloc(256);
    status.alloc(1);
    CK(cudaMemsetAsync(status.p, 0, sizeof(unsigned), st));
    rho_plane.alloc(nr);
  }
  ~EngineT() override {
    if (pin) cudaFreeHost(pin);
    if (step_exec) cudaGraphExecDestroy(step_exec);
    for (cudaEvent_t e : hev) cudaEventDestroy(e);
    if (hcs) cudaStreamDestroy(hcs);
  }

  Sub<T>& sub(int i) {
    REQ(i >= 0 && i < (int)subs.size(), FDE_EINVAL, "subsystem index out of range");
    return *subs[i];
  }
  int nsub() const override { return (int)subs.size(); }
  long long grid_points() const override { return nr; }
  void shape(int i, int* nb, int* nk) override {
    *nb = sub(i).nb;
    *nk = sub(i).nk;
  }
  int npw(int i, int k) override { return kpt(i, k).npw; }
  void set_eig_occ(int i, int k, const double* eig, const double* occ) override {
    KP<T>& q = kpt(i, k);
    const int nb = sub(i).nb;
    q.eig.assign(eig, eig + nb);
    q.occ.assign(occ, occ + nb);
    q.have_eig = true;
  }
  void set_subsystem_entropy(int i, double ts) override { sub(i).entropy = ts; }
  double subsystem_entropy(int i) override { return sub(i).entropy; }
  KP<T>& kpt(int i, int k) {
    Sub<T>& s = sub(i);
    REQ(k >= 0 && k < s.nk, FDE_EINVAL, "k-point index out of range");
    return s.kp[k];
  }
  void fft3d(void* data, int sign) override {
    REQ(data && (sign == 1 || sign == -1), FDE_EINVAL, "bad transform arguments");
    C* d = (C*)data;
    launch_fft3d<T>(d, g, plans.fp, sign, st);
    if (sign < 0) grid_scale_c<T>(d, 1.0 / (double)nr, nr, st);
  }
  // The potential build's transform of an FP64 grid: arith 0 FP64, 1 double-float.
  void fft3d_f64(double2* data, int sign, int arith) override {
    REQ(data && (sign == 1 || sign == -1) && (arith == 0 || arith == 1), FDE_EINVAL, "bad transform arguments");
    if (arith == 1) {
      if constexpr (sizeof(T) == 4) {
        REQ(launch_fft3d_dd(data, g, plansdd.fp, sign, st), FDE_EUNSUPPORTED, "no double-float kernel for a length");
      } else {
        Plans<dd> p;
        make_plans(p, grid, st);
        REQ(launch_fft3d_dd(data, g, p.fp, sign, st), FDE_EUNSUPPORTED, "no double-float kernel for a length");
        CK(cudaStreamSynchronize(st));  // p's tables are released on return
      }
    } else {
      launch_fft3d<double>(data, g, plans64.fp, sign, st);
    }
    if (sign < 0) grid_scale_c<double>(data, 1.0 / (double)nr, nr, st);
  }
  void sync() override {
    CK(cudaStreamSynchronize(st));
    unsigned h = 0;
    CK(cudaMemcpy(&h, status.p, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (h & ST_NONFINITE) {
      CK(cudaMemset(status.p, 0, sizeof(unsigned)));
      throw Err{FDE_ENONFINITE, "non-finite value on the device"};
    }
    if (sizeof(T) == 4 && (gemm_tc_take_status(st) & ST_TIMEOUT))
      throw Err{FDE_ETIMEOUT, "a tensor-core product timed out waiting for its MMAs"};
    if (precond_tc_take_status(st) & ST_TIMEOUT)
      throw Err{FDE_ETIMEOUT, "the learned preconditioner's tensor-core inference timed out"};
  }

  // ---- basis ------------------------------------------------------------------------------
  void build_sphere(KP<T>& q) {
    const double Lc[3] = {A[0][0], A[1][1], A[2][2]};
    sphere_miller(Lc, q.kfrac, ecut, q.miller, q.kin, q.kc);
    q.npw = (int)q.kin.size();
    REQ(q.npw > 0, FDE_EINVAL, "empty plane-wave sphere");
    for (int j = 0; j < 3; ++j) {
      int lo = 1 << 30, hi = -(1 << 30);
      for (int p = 0; p < q.npw; ++p) { lo = std::min(lo, q.miller[3 * p + j]); hi = std::max(hi, q.miller[3 * p + j]); }
      REQ(hi - lo + 1 <= grid[j], FDE_EINVAL, "plane-wave sphere does not fit the grid");
    }
    // columns (m1, m2) with contiguous m3 runs (enumeration order is already sorted)
    std::vector<int> cs, m3lo, ci1, ci2;
    for (int p = 0; p < q.npw; ++p) {
      const int m1 = q.miller[3 * p], m2 = q.miller[3 * p + 1];
      if (p == 0 || m1 != q.miller[3 * (p - 1)] || m2 != q.miller[3 * (p - 1) + 1]) {
        cs.push_back(p);
        m3lo.push_back(q.miller[3 * p + 2]);
        ci1.push_back(((m1 % grid[0]) + grid[0]) % grid[0]);
        ci2.push_back(((m2 % grid[1]) + grid[1]) % grid[1]);
      }
    }
    const int ncol = (int)m3lo.size();
    cs.push_back(q.npw);
    std::vector<int> rows;
    for (int c = 0; c < ncol; ++c)
      if (std::find(rows.begin(), rows.end(), ci1[c]) == rows.end()) rows.push_back(ci1[c]);
    std::vector<int> all;
    all.insert(all.end(), cs.begin(), cs.end());
    all.insert(all.end(), m3lo.begin(), m3lo.end());
    all.insert(all.end(), ci1.begin(), ci1.end());
    all.insert(all.end(), ci2.begin(), ci2.end());
    all.insert(all.end(), rows.begin(), rows.end());
    q.cols.alloc(all.size());
    CK(cudaMemcpy(q.cols.p, all.data(), all.size() * sizeof(int), cudaMemcpyHostToDevice));
    q.sp.npw = q.npw;
    q.sp.ncol = ncol;
    q.sp.nrow = (int)rows.size();
    q.sp.col_start = q.cols.p;
    q.sp.col_m3lo = q.cols.p + (ncol + 1);
    q.sp.col_i1 = q.cols.p + (2 * ncol + 1);
    q.sp.col_i2 = q.cols.p + (3 * ncol + 1);
    q.sp.row_i1 = q.cols.p + (4 * ncol + 1);
    std::vector<T> kt(q.npw);
    for (int p = 0; p < q.npw; ++p) kt[p] = (T)q.kin[p];
    q.kin_d.alloc(q.npw);
    CK(cudaMemcpy(q.kin_d.p, kt.data(), q.npw * sizeof(T), cudaMemcpyHostToDevice));
  }

  void build_projectors(Sub<T>& s, KP<T>& q) {
    if (s.nproj == 0) return;
    std::vector<C> h((size_t)s.nproj * q.npw);
    for (int p = 0; p < q.npw; ++p) {
      double qv[3];
      for (int c = 0; c < 3; ++c)
        qv[c] = q.kc[c] + ((double)q.miller[3 * p] * B[0][c] + (double)q.miller[3 * p + 1] * B[1][c] +
                           (double)q.miller[3 * p + 2] * B[2][c]);
      const double q2 = qv[0] * qv[0] + qv[1] * qv[1] + qv[2] * qv[2];
      for (int a = 0; a < s.natoms; ++a) {
        const double ph = qv[0] * s.pos[3 * a] + qv[1] * s.pos[3 * a + 1] + qv[2] * s.pos[3 * a + 2];
        const double cr = cos(ph), ci = -sin(ph);
        for (int i = 0; i < s.nproj_atom; ++i) {
          const double sg = s.sigma[i];
          const double amp = pow(omega, -0.5) * pow(pow(M_PI, 1.5) * sg * sg * sg, -0.5) * pow(2.0 * M_PI * sg * sg, 1.5) *
                             exp(-q2 * sg * sg / 2.0);
          h[(size_t)(a * s.nproj_atom + i) * q.npw + p] = mk<T>((T)(amp * cr), (T)(amp * ci));
        }
      }
    }
    q.beta.alloc(h.size());
    CK(cudaMemcpy(q.beta.p, h.data(), h.size() * sizeof(C), cudaMemcpyHostToDevice));
  }

  int add_subsystem(const fde_subsys_desc* d) override {
    REQ(d, FDE_EINVAL, "null subsystem descriptor");
    REQ(!locked, FDE_EINVAL, "subsystems must be added before the potentials are built");
    REQ(d->natoms >= 0 && d->nbands > 0 && d->nk > 0, FDE_EINVAL, "bad subsystem sizes");
    REQ(d->natoms == 0 || (d->pos && d->Z), FDE_EINVAL, "null atom arrays");
    REQ(d->kpts && d->wk, FDE_EINVAL, "null k-point arrays");
    REQ(d->nproj_per_atom >= 0 && (d->nproj_per_atom == 0 || (d->proj_sigma && d->proj_D)), FDE_EINVAL,
        "null projector arrays");
    REQ(d->nproj_per_atom <= 8, FDE_EUNSUPPORTED, "at most 8 projectors per atom");
    if (d->smearing_ha <= 0) {
      const double no = d->nelec / 2.0;
      REQ(d->nk == 1 && fabs(no - round(no)) < 1e-12 && round(no) <= d->nbands && no >= 0, FDE_EINVAL,
          "integer occupations need one k-point and nelec/2 <= nbands");
    }
    auto s = std::make_unique<Sub<T>>();
    s->natoms = d->natoms;
    s->nproj_atom = d->nproj_per_atom;
    s->nproj = d->natoms * d->nproj_per_atom;
    s->nb = d->nbands;
    s->nk = d->nk;
    s->rc = d->rc;
    s->nelec = d->nelec;
    s->smearing = d->smearing_ha;
    REQ(d->smearing_kind == FDE_SMEAR_FERMI || d->smearing_kind == FDE_SMEAR_MP || d->smearing_kind == FDE_SMEAR_GAUSS,
        FDE_EINVAL, "unknown smearing kind");
    s->smear_kind = d->smearing_kind;
    s->pos.assign(d->pos, d->pos + 3 * d->natoms);
    s->Z.assign(d->Z, d->Z + d->natoms);
    if (s->nproj_atom) {
      s->sigma.assign(d->proj_sigma, d->proj_sigma + s->nproj_atom);
      s->D.assign(d->proj_D, d->proj_D + s->nproj_atom * s->nproj_atom);
    }
    s->kpts.assign(d->kpts, d->kpts + 3 * d->nk);
    s->wk.assign(d->wk, d->wk + d->nk);
    if (!subs.empty()) REQ(subs[0]->rc == s->rc, FDE_EINVAL, "one r_c for every atom");
    s->kp.resize(s->nk);
    for (int k = 0; k < s->nk; ++k) {
      KP<T>& q = s->kp[k];
      for (int c = 0; c < 3; ++c) q.kfrac[c] = s->kpts[3 * k + c];
      build_sphere(q);
      build_projectors(*s, q);
      q.X.alloc((size_t)s->nb * q.npw);
      q.HX.alloc((size_t)s->nb * q.npw);
      q.eig.assign(s->nb, 0.0);
      q.occ.assign(s->nb, 0.0);
    }
    if (s->nproj) {
      s->Dblk.np = s->nproj_atom;
      for (int i = 0; i < s->nproj_atom * s->nproj_atom; ++i) s->Dblk.d[i] = s->D[i];
    }
    if (d->aug_sigma > 0) {
      REQ(s->nproj > 0 && d->proj_Q, FDE_EINVAL, "augmentation needs projectors and their q matrix");
      s->uspp = true;
      s->aug_sigma = d->aug_sigma;
      s->Q.assign(d->proj_Q, d->proj_Q + s->nproj_atom * s->nproj_atom);
      s->Qblk.np = s->nproj_atom;
      for (int i = 0; i < s->nproj_atom * s->nproj_atom; ++i) s->Qblk.d[i] = s->Q[i];
      s->aug_pos.alloc(3 * (size_t)s->natoms);
      CK(cudaMemcpy(s->aug_pos.p, s->pos.data(), 3 * (size_t)s->natoms * sizeof(double), cudaMemcpyHostToDevice));
      // the screened couplings start as the bare one (until the first potential)
      std::vector<double> d0((size_t)s->natoms * s->nproj_atom * s->nproj_atom);
      for (int a = 0; a < s->natoms; ++a)
        std::copy(s->D.begin(), s->D.end(), d0.begin() + (size_t)a * s->nproj_atom * s->nproj_atom);
      s->Dscr.alloc(d0.size());
      CK(cudaMemcpy(s->Dscr.p, d0.data(), d0.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
    s->rho.alloc(nr);
    s->veff.alloc(nr);
    s->vplane.alloc(nr);
    CK(cudaMemsetAsync(s->rho.p, 0, nr * sizeof(double), st));
    CK(cudaMemsetAsync(s->veff.p, 0, nr * sizeof(double), st));
    CK(cudaMemsetAsync(s->vplane.p, 0, nr * sizeof(T), st));
    subs.push_back(std::move(s));
    return (int)subs.size() - 1;
  }

  void get_basis(int i, int k, int* npw, int* miller) override {
    KP<T>& q = kpt(i, k);
    REQ(npw, FDE_EINVAL, "null npw");
    *npw = q.npw;
    if (miller) memcpy(miller, q.miller.data(), q.miller.size() * sizeof(int));
  }

  // ---- local potential of all nuclei and nuclear repulsion (once per geometry) -----------------
  void ensure_vloc() {
    if (locked) return;
    REQ(!subs.empty(), FDE_EINVAL, "no subsystems");
    std::vector<double> pos, Z;
    for (auto& s : subs) {
      pos.insert(pos.end(), s->pos.begin(), s->pos.end());
      Z.insert(Z.end(), s->Z.begin(), s->Z.end());
    }
    vloc.alloc(nr);
    cvl.alloc(nr);
    const int na = (int)Z.size();
    DBuf<double> dp, dz;
    dp.alloc(std::max(1, 3 * na));
    dz.alloc(std::max(1, na));
    if (na) {
      CK(cudaMemcpyAsync(dp.p, pos.data(), 3 * na * sizeof(double), cudaMemcpyHostToDevice, st));
      CK(cudaMemcpyAsync(dz.p, Z.data(), na * sizeof(double), cudaMemcpyHostToDevice, st));
    }
    grid_vloc_g(cvl.p, g, cell, dp.p, dz.p, na, subs[0]->rc, st);
    launch_fft3d<double>(cvl.p, g, plans64.fp, +1, st);
    grid_c_to_real<double>(cvl.p, vloc.p, nr, st);
    CK(cudaStreamSynchronize(st));
    cvl.release();
    const double Lc[3] = {A[0][0], A[1][1], A[2][2]};
    enn = ewald_energy(Lc, pos, Z);
    locked = true;
  }

  // ---- densities ----------------------------------------------------------------------------
  void set_density(int i, const double* rho, int on_device) override {
    REQ(rho, FDE_EINVAL, "null density");
    Sub<T>& s = sub(i);
    CK(cudaMemcpyAsync(s.rho.p, rho, nr * sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    // a pageable source is read when the copy is issued, a page-locked one later by the copy
    // engine: the caller may reuse its buffer once the call returns in both cases
    if (!on_device) CK(cudaStreamSynchronize(st));
  }
  void sum_densities() {
    CK(cudaMemcpyAsync(rho_tot.p, subs[0]->rho.p, nr * sizeof(double), cudaMemcpyDeviceToDevice, st));
    for (size_t I = 1; I < subs.size(); ++I)
      grid_combine<double>(rho_tot.p, subs[I]->rho.p, nullptr, nullptr, 0.0, rho_tot.p, nr, st);
  }
  void get_density(int i, double* d_rho) override {
    REQ(d_rho, FDE_EINVAL, "null output");
    if (i == -1) {
      REQ(!subs.empty(), FDE_EINVAL, "no subsystems");
      sum_densities();
      CK(cudaMemcpyAsync(d_rho, rho_tot.p, nr * sizeof(double), cudaMemcpyDeviceToDevice, st));
    } else {
      CK(cudaMemcpyAsync(d_rho, sub(i).rho.p, nr * sizeof(double), cudaMemcpyDeviceToDevice, st));
    }
  }

  // ---- embedding-potential build --------------------------------------------------------------
  bool gga_xc() const { return func.xc == FDE_XC_PBE; }
  bool gga_kin() const { return func.kedf != FDE_KEDF_TF; }

  // Transforms of the densities and their gradients (FP64 grids): FP64 arithmetic in FP64
  // contexts; double-float arithmetic on the FP32 pipes (~48 bits) in mixed ones.
  void fft_density(double2* x, int sign) {
    if constexpr (sizeof(T) == 4) {
      if (launch_fft3d_dd(x, g, plansdd.fp, sign, st)) return;
    }
    launch_fft3d<double>(x, g, plans64.fp, sign, st);
  }

  // Divergence-argument grid c of pair q in the working precision: the packed gradient grid
  // itself (overwritten in place) in FP64 contexts, a separate FP32 grid in mixed ones.
  std::vector<DBuf<cplx<T>>> dpacks;
  DBuf<cplx<T>> fpot;
  cplx<T>* dgrid(int q, int c, double2* packed) {
    if constexpr (sizeof(T) == 8) {
      return reinterpret_cast<cplx<T>*>(packed);
    } else {
      const size_t need = (size_t)3 * (q + 1);
      if (dpacks.size() < need) dpacks.resize(need);
      DBuf<cplx<T>>& b = dpacks[(size_t)3 * q + c];
      if (!b.p) b.alloc(nr);
      return b.p;
    }
  }
  // Reciprocal-space potentials of a pair (the packed transform grid in FP64 contexts).
  cplx<T>* fgrid() {
    if constexpr (sizeof(T) == 8) {
      return reinterpret_cast<cplx<T>*>(cb[0].p);
    } else {
      if (!fpot.p) fpot.alloc(nr);
      return fpot.p;
    }
  }

  // Packed gradient grids of subsystem pair q (three complex grids).
  double2* pack(int q, int c) {
    const size_t need = (size_t)3 * (q + 1);
    if (packs.size() < need) packs.resize(need);
    DBuf<double2>& b = packs[(size_t)3 * q + c];
    if (!b.p) b.alloc(nr);
    return b.p;
  }

  // Builds the potentials (want_pot) of the subsystems in `which` (-1 all) and/or the grid
  // energy terms (want_e); slots of scal: 0 E_H, 1/2 E_xc/T_tot, 3 E_loc, then per
  // subsystem 4+3I: E_H[rho_I], 5+3I: E_xc[rho_I], 6+3I: T[rho_I].
  //
  // v_eff^I = v_loc + v_H[rho] + v_xc[rho] + v~_kin[rho] - v~_kin[rho_I] (Eq. 4 with the
  // kinetic potential of Eq. 7): with f the pointwise energy densities, a functional's
  // potential is df/drho - div(df/dgrad rho), so
  //   v_eff^I = v_loc + v_H + (w_tot - w_I) - div(h_tot - h_I)
  // where w and h are the two derivatives at rho (xc + kinetic) and at rho_I (kinetic).
  // Subsystems are taken in pairs (a, b), each pair's real fields packed into one complex
  // transform: rho_a + i rho_b forward, the gradients as (x + i y of a), (x + i y of b),
  // (z of a + i z of b) backward, the divergence arguments the same way forward, and
  // (v_a + i v_b) backward: 8 transforms per pair.
  EnergyParts grid_pass(bool want_pot, bool want_e, int which) {
    ensure_vloc();
    REQ(4 + 3 * subs.size() <= 250, FDE_EUNSUPPORTED, "too many subsystems for one energy pass");
    const int nsb = (int)subs.size();
    const int npairs = (nsb + 1) / 2;
    REQ(npairs <= kMaxPairs, FDE_EUNSUPPORTED, "at most 64 subsystems");
    const size_t nrb = (size_t)grid_red_blocks();
    const double dv = omega / (double)nr;
    const bool grad = gga_xc() || gga_kin();
    double2* C = cb[0].p;
    double2* RT = cb[1].p;
    sum_densities();
    // 1. densities to reciprocal space, total density, Hartree sums and gradients
    GradPacks gp{};
    gp.npairs = grad ? npairs : 0;
    for (int q = 0; q < npairs; ++q) {
      const int ia = 2 * q, ib = 2 * q + 1;
      const bool hb = ib < nsb;
      grid_pack2(subs[ia]->rho.p, hb ? subs[ib]->rho.p : nullptr, C, nr, st);
      fft_density(C, -1);
      double2* Pa = grad ? pack(q, 0) : nullptr;
      double2* Pb = (grad && hb) ? pack(q, 1) : nullptr;
      double2* Pz = grad ? pack(q, 2) : nullptr;
      grid_unpack_density(C, hb ? 1 : 0, RT, q > 0 ? 1 : 0, Pa, Pb, Pz, g, cell, want_e ? partial.p : nullptr, st);
      if (want_e) {
        grid_finalize(partial.p, 1, 0.5 * omega, scal.p + 4 + 3 * ia, st);
        if (hb) grid_finalize(partial.p + nrb, 1, 0.5 * omega, scal.p + 4 + 3 * ib, st);
      }
      if (grad) {
        fft_density(Pa, +1);
        if (hb) fft_density(Pb, +1);
        fft_density(Pz, +1);
        gp.a[q] = Pa;
        gp.b[q] = Pb;
        gp.z[q] = Pz;
        gp.has_b[q] = hb ? 1 : 0;
      }
    }
    // 2. functionals of the total density
    grid_pw_total(rho_tot.p, gp, func.xc, func.kedf, func.rho_cut, want_pot ? vpart.p : nullptr,
                  (want_pot && grad) ? htot[0].p : nullptr, htot[1].p, htot[2].p, nr, partial.p, sizeof(T) == 4,
                  st);
    if (want_e) {  // the pointwise kernels always leave their block sums; reduce them only when asked
      grid_finalize(partial.p, 2, dv, scal.p + 1, st);
      grid_dot_partial(vloc.p, rho_tot.p, nr, 0, partial.p, st);
      grid_finalize(partial.p, 1, dv, scal.p + 3, st);
    }
    if (want_e) {
      grid_assemble_pair<double>(RT, nullptr, nullptr, nullptr, 0, nullptr, g, cell, partial.p, st);
      grid_finalize(partial.p, 1, 0.5 * omega, scal.p + 0, st);
    }
    // 3. per pair: subsystem functionals, divergences, reciprocal-space part, potentials
    for (int q = 0; q < npairs; ++q) {
      const int ia = 2 * q, ib = 2 * q + 1;
      const bool hb = ib < nsb;
      const bool pa = want_pot && (which < 0 || which == ia);
      const bool pb = hb && want_pot && (which < 0 || which == ib);
      if (!pa && !pb && !want_e) continue;
      Sub<T>& A = *subs[ia];
      Sub<T>* B = hb ? subs[ib].get() : nullptr;
      double2* Pa = grad ? pack(q, 0) : nullptr;
      double2* Pb = (grad && hb) ? pack(q, 1) : nullptr;
      double2* Pz = grad ? pack(q, 2) : nullptr;
      const bool pot = pa || pb;
      // divergence arguments, reciprocal-space potentials and their transforms in the working
      // precision (FP32 in mixed contexts: they enter V_eff linearly, unlike the gradients)
      cplx<T>* Da = grad ? dgrid(q, 0, Pa) : nullptr;
      cplx<T>* Db = (grad && hb) ? dgrid(q, 1, Pb) : nullptr;
      cplx<T>* Dz = grad ? dgrid(q, 2, Pz) : nullptr;
      cplx<T>* F = fgrid();
      grid_pw_pair<T>(A.rho.p, B ? B->rho.p : nullptr, Pa, Pb, Pz, Da, Db, Dz, htot[0].p, htot[1].p, htot[2].p,
                      want_pot ? vpart.p : nullptr, want_e ? func.xc : -1, func.kedf, func.rho_cut,
                      pa ? A.veff.p : nullptr, pb ? B->veff.p : nullptr, (pot && grad) ? 1 : 0, nr, partial.p, st);
      if (want_e) {
        grid_finalize(partial.p, 2, dv, scal.p + 5 + 3 * ia, st);
        if (hb) grid_finalize(partial.p + 2 * nrb, 2, dv, scal.p + 5 + 3 * ib, st);
      }
      if (!pot) continue;
      if (grad) {
        launch_fft3d<T>(Da, g, plans.fp, -1, st);
        if (hb) launch_fft3d<T>(Db, g, plans.fp, -1, st);
        launch_fft3d<T>(Dz, g, plans.fp, -1, st);
      }
      grid_assemble_pair<T>(RT, Da, Db, Dz, hb ? 1 : 0, F, g, cell, nullptr, st);
      launch_fft3d<T>(F, g, plans.fp, +1, st);
      grid_finish_pair<T>(F, vloc.p, pa ? A.veff.p : nullptr, pb ? B->veff.p : nullptr, nr, st);
      if (pa) {
        grid_nonfinite(A.veff.p, nr, status.p, st);
        to_plane(A);
        refresh_screening(A);
      }
      if (pb) {
        grid_nonfinite(B->veff.p, nr, status.p, st);
        to_plane(*B);
        refresh_screening(*B);
      }
    }
    EnergyParts ep;
    if (want_e) {
      std::vector<double> h(4 + 3 * subs.size());
      CK(cudaMemcpyAsync(h.data(), scal.p, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
      sync();
      ep.EH = h[0];
      ep.Exc = h[1];
      ep.Ttot = h[2];
      ep.Eloc = h[3];
      for (size_t I = 0; I < subs.size(); ++I) {
        ep.EH_sub += h[4 + 3 * I];
        ep.Exc_sub += h[5 + 3 * I];
        ep.Tsub += h[6 + 3 * I];
      }
    }
    return ep;
  }
  void neg_add(double* a, const double* b) { grid_axpy(a, b, -1.0, nr, st); }
  // Plane-major copy of V_eff^I in the working precision for the plane pass of H psi:
  // [i3][i1][i2].
  void to_plane(Sub<T>& s) {
    launch_transpose<double, T>(s.veff.p, s.vplane.p, (int)((long long)g.n1 * g.n2), g.n3, 0, st);
  }

  void build_vemb(double* d_out, fde_energies* e) override {
    ensure_vloc();
    EnergyParts ep = grid_pass(true, e != nullptr, -1);
    if (d_out)
      for (size_t I = 0; I < subs.size(); ++I)
        CK(cudaMemcpyAsync(d_out + I * nr, subs[I]->veff.p, nr * sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (e) {
      memset(e, 0, sizeof(*e));
      e->E_loc = ep.Eloc;
      e->E_H = ep.EH;
      e->E_xc = ep.Exc;
      e->T_nad = ep.Ttot - ep.Tsub;
      e->E_xc_nad = ep.Exc - ep.Exc_sub;
      e->E_H_nad = ep.EH - ep.EH_sub;
      e->E_nn = enn;
    }
  }

  void set_veff(int i, const double* d_v) override {
    REQ(d_v, FDE_EINVAL, "null potential");
    Sub<T>& s = sub(i);
    CK(cudaMemcpyAsync(s.veff.p, d_v, nr * sizeof(double), cudaMemcpyDeviceToDevice, st));
    to_plane(s);
    refresh_screening(s);
  }

  // Screened couplings of an ultrasoft-like subsystem from its current V_eff^I:
  // D_a = D + q int V_eff^I g_a, the integral by Parseval against V_eff^I's transform.
  void refresh_screening(Sub<T>& s) {
    if (!s.uspp) return;
    double2* C = cb[0].p;
    grid_pack2(s.veff.p, nullptr, C, nr, st);
    launch_fft3d<double>(C, g, plans64.fp, -1, st);
    grid_scale_c<double>(C, 1.0 / (double)nr, nr, st);
    grid_aug_screening(C, g, cell, s.aug_pos.p, s.natoms, s.aug_sigma, s.Dblk, s.Qblk, s.Dscr.p, st);
  }

  // S_I psi = psi + sum_{a in I} beta q <beta|psi> (a copy of psi for norm-conserving I).
  void apply_s(Sub<T>& s, KP<T>& q, const C* psi, C* spsi, int nb) {
    CK(cudaMemcpyAsync(spsi, psi, (size_t)nb * q.npw * sizeof(C), cudaMemcpyDeviceToDevice, st));
    if (!s.uspp) return;
    gwork.ensure(gemm_hn_work(s.nproj, nb, q.npw));
    Pm.ensure((size_t)s.nproj * nb);
    Qm.ensure((size_t)s.nproj * nb);
    launch_gemm_hn<T>(q.beta.p, q.npw, psi, q.npw, s.nproj, nb, q.npw, Pm.p, nb, gwork.p, st);
    launch_kb_couple(Pm.p, s.Qblk, s.natoms, nb, Qm.p, st);
    launch_gemm_rot<T>(q.beta.p, q.npw, Qm.p, nb, s.nproj, nb, q.npw, spsi, q.npw, 1.0, 1.0, st);
  }

  // ---- H psi ----------------------------------------------------------------------------------
  long long davidson_iters = 0, hpsi_bands = 0;
  void apply_h_dev(Sub<T>& s, KP<T>& q, const C* psi, C* hpsi, int nb) {
    hpsi_bands += nb;
    scratch.ensure((size_t)nb * g.n3 * q.sp.ncol);
    launch_hpsi_local<T>(psi, q.npw, hpsi, q.npw, nb, q.kin_d.p, s.vplane.p, scratch.p, q.sp, g, plans.fp, st);
    apply_nl(s, q, psi, hpsi, nb);
  }
  // hpsi += sum_{a in I} beta D <beta|psi> (projectors of the subsystem's own atoms)
  void apply_nl(Sub<T>& s, KP<T>& q, const C* psi, C* hpsi, int nb) {
    if (s.nproj) {
      gwork.ensure(gemm_hn_work(s.nproj, nb, q.npw));
      Pm.ensure((size_t)s.nproj * nb);
      Qm.ensure((size_t)s.nproj * nb);
      launch_gemm_hn<T>(q.beta.p, q.npw, psi, q.npw, s.nproj, nb, q.npw, Pm.p, nb, gwork.p, st);
      if (s.uspp) launch_kb_couple_atoms(Pm.p, s.Dscr.p, s.nproj_atom, s.natoms, nb, Qm.p, st);
      else launch_kb_couple(Pm.p, s.Dblk, s.natoms, nb, Qm.p, st);
      launch_gemm_rot<T>(q.beta.p, q.npw, Qm.p, nb, s.nproj, nb, q.npw, hpsi, q.npw, 1.0, 1.0, st);
    }
  }
  void apply_h(int i, int k, const void* psi, void* hpsi, int nb) override {
    REQ(psi && hpsi, FDE_EINVAL, "null orbital buffers");
    REQ(nb > 0, FDE_EINVAL, "nb must be positive");
    Sub<T>& s = sub(i);
    KP<T>& q = kpt(i, k);
    apply_h_dev(s, q, (const C*)psi, (C*)hpsi, nb);
  }
  // True if the host range [p, p + bytes) lies in page-locked memory the copy engines can
  // read directly (allocated with cudaHostAlloc / cudaMallocHost or registered).
  static bool host_pinned(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
      cudaGetLastError();  // clear the error of a plain pageable pointer
      return false;
    }
    return a.type == cudaMemoryTypeHost;
  }
  void apply_s_dev(int i, int k, const void* psi, void* spsi, int nb) override {
    REQ(psi && spsi && nb > 0, FDE_EINVAL, "bad orbital buffers");
    apply_s(sub(i), kpt(i, k), (const C*)psi, (C*)spsi, nb);
  }
  void apply_h_host(int i, int k, const double* psi, double* hpsi, int nb) override {
    REQ(psi && hpsi && nb > 0, FDE_EINVAL, "bad host buffers");
    Sub<T>& s = sub(i);
    KP<T>& q = kpt(i, k);
    const size_t n = (size_t)nb * q.npw;
    if (host_pinned(psi) && host_pinned(hpsi)) {
      // page-locked caller buffers: the copy engines move them directly, no staging
      V.ensure(n);
      V2.ensure(n);
      DBuf<double2>& d64 = S;
      d64.ensure(n);
      CK(cudaMemcpyAsync(d64.p, psi, n * sizeof(double2), cudaMemcpyHostToDevice, st));
      convert_in(d64.p, V.p, n);
      apply_h_dev(s, q, V.p, V2.p, nb);
      convert_out(V2.p, d64.p, n);
      CK(cudaMemcpyAsync(hpsi, d64.p, n * sizeof(double2), cudaMemcpyDeviceToHost, st));
      sync();
      return;
    }
    if (pin_n < 2 * n) {
      if (pin) cudaFreeHost(pin);
      pin = nullptr;
      CK(cudaMallocHost(&pin, 2 * n * sizeof(double2)));
      pin_n = 2 * n;
    }
    V.ensure(n);
    V2.ensure(n);
    DBuf<double2>& d64 = S;  // staging in FP64 complex
    d64.ensure(n);
    memcpy(pin, psi, n * sizeof(double2));
    CK(cudaMemcpyAsync(d64.p, pin, n * sizeof(double2), cudaMemcpyHostToDevice, st));
    convert_in(d64.p, V.p, n);
    apply_h_dev(s, q, V.p, V2.p, nb);
    convert_out(V2.p, d64.p, n);
    CK(cudaMemcpyAsync(pin + 2 * n, d64.p, n * sizeof(double2), cudaMemcpyDeviceToHost, st));
    sync();
    memcpy(hpsi, pin + 2 * n, n * sizeof(double2));
  }
  void convert_in(const double2* a, C* b, size_t n);
  void convert_out(const C* a, double2* b, size_t n);

  // H psi of every band of every (subsystem, k): the local part of all of them in one
  // batched launch per phase, then each subsystem's own projectors.
  void apply_h_all() override {
    size_t total = 0;
    for (auto& sp : subs)
      for (auto& q : sp->kp) total += (size_t)sp->nb * g.n3 * q.sp.ncol;
    scratch.ensure(total);
    std::vector<HpsiItemDesc<T>> items;
    size_t off = 0;
    for (auto& sp : subs)
      for (auto& q : sp->kp) {
        items.push_back(HpsiItemDesc<T>{q.sp, q.X.p, q.HX.p, q.kin_d.p, sp->vplane.p, scratch.p + off, q.npw, sp->nb});
        off += (size_t)sp->nb * g.n3 * q.sp.ncol;
      }
    if (!launch_hpsi_batch_ct<T>(items.data(), (int)items.size(), g, plans.fp, st)) {
      for (auto& sp : subs)
        for (auto& q : sp->kp) apply_h_dev(*sp, q, q.X.p, q.HX.p, sp->nb);
      return;
    }
    for (auto& sp : subs)
      for (auto& q : sp->kp) {
        hpsi_bands += sp->nb;
        apply_nl(*sp, q, q.X.p, q.HX.p, sp->nb);
      }
  }

  // One pass of the hot path with host buffers: every subsystem density and every (subsystem,
  // k) orbital block in, every H psi block out.  The orbital blocks go up on a copy stream
  // while the context stream uploads the densities and builds the potentials; each block is
  // converted to the working precision once its copy has landed, all bands go through the
  // batched H psi, and the results come back block by block.  The blocks replace the stored
  // orbitals.  Synchronising.
  cudaStream_t hcs = nullptr;
  std::vector<cudaEvent_t> hev;
  DBuf<double2> hstage;  // FP64 images of every block, end to end (orbitals in, then H psi out)
  void hot_step_host(const double* const* rho, const double* const* psi, double* const* hpsi) override {
    REQ(rho && psi && hpsi, FDE_EINVAL, "null host buffer table");
    REQ(!subs.empty(), FDE_EINVAL, "no subsystems");
    ensure_vloc();
    std::vector<size_t> off;
    size_t tot = 0;
    for (auto& sp : subs)
      for (auto& q : sp->kp) {
        REQ(psi[off.size()] && hpsi[off.size()], FDE_EINVAL, "null orbital block");
        off.push_back(tot);
        tot += (size_t)sp->nb * q.npw;
      }
    for (size_t I = 0; I < subs.size(); ++I) REQ(rho[I], FDE_EINVAL, "null density");
    const int nblk = (int)off.size();
    hstage.ensure(tot);
    if (!hcs) CK(cudaStreamCreateWithFlags(&hcs, cudaStreamNonBlocking));
    while ((int)hev.size() < nblk + 1) {
      cudaEvent_t e;
      CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      hev.push_back(e);
    }
    // the staging buffer is free once the context stream's earlier work (a previous call's
    // output copies) is done
    CK(cudaEventRecord(hev[nblk], st));
    CK(cudaStreamWaitEvent(hcs, hev[nblk], 0));
    int b = 0;
    for (auto& sp : subs)
      for (auto& q : sp->kp) {
        CK(cudaMemcpyAsync(hstage.p + off[b], psi[b], (size_t)sp->nb * q.npw * sizeof(double2),
                           cudaMemcpyHostToDevice, hcs));
        CK(cudaEventRecord(hev[b], hcs));
        ++b;
      }
    for (size_t I = 0; I < subs.size(); ++I)
      CK(cudaMemcpyAsync(subs[I]->rho.p, rho[I], nr * sizeof(double), cudaMemcpyHostToDevice, st));
    grid_pass(true, false, -1);
    b = 0;
    for (auto& sp : subs)
      for (auto& q : sp->kp) {
        CK(cudaStreamWaitEvent(st, hev[b], 0));
        convert_in(hstage.p + off[b], q.X.p, (size_t)sp->nb * q.npw);
        q.have_orbitals = true;
        q.have_eig = false;
        ++b;
      }
    apply_h_all();
    b = 0;
    for (auto& sp : subs)
      for (auto& q : sp->kp) {
        const size_t n = (size_t)sp->nb * q.npw;
        convert_out(q.HX.p, hstage.p + off[b], n);
        CK(cudaMemcpyAsync(hpsi[b], hstage.p + off[b], n * sizeof(double2), cudaMemcpyDeviceToHost, st));
        ++b;
      }
    sync();
  }

  // One pass of the hot path over the whole cell (potential build + every band's H psi),
  // optionally replayed from a captured CUDA graph.
  cudaGraphExec_t step_exec = nullptr;
  unsigned long long step_gen = ~0ull;
  long long step_kernels = 0;
  void hot_step(bool use_graph) override {
    ensure_vloc();
    if (!use_graph) {
      grid_pass(true, false, -1);
      apply_h_all();
      return;
    }
    if (!step_exec || step_gen != g_alloc_generation) {
      grid_pass(true, false, -1);  // an eager pass sizes every buffer first
      apply_h_all();
      CK(cudaStreamSynchronize(st));
      if (step_exec) {
        cudaGraphExecDestroy(step_exec);
        step_exec = nullptr;
      }
      Profiler* pr = tl_prof;
      const long long before = pr ? pr->launches : 0;
      const bool was_on = pr && pr->on;
      if (pr) pr->on = false;
      cudaGraph_t gph;
      CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      grid_pass(true, false, -1);
      apply_h_all();
      CK(cudaStreamEndCapture(st, &gph));
      const cudaError_t ie = cudaGraphInstantiate(&step_exec, gph, 0);
      cudaGraphDestroy(gph);
      CK(ie);
      step_kernels = pr ? pr->launches - before : 0;
      if (pr) {
        pr->on = was_on;
        pr->launches = before;
      }
      step_gen = g_alloc_generation;
    }
    CK(cudaGraphLaunch(step_exec, st));
    if (tl_prof) tl_prof->launches += step_kernels;
  }

  // ---- orbitals -------------------------------------------------------------------------------
  void init_orbitals(int i, int k, const double* raw) override {
    REQ(raw, FDE_EINVAL, "null raw draws");
    Sub<T>& s = sub(i);
    KP<T>& q = kpt(i, k);
    const size_t n = (size_t)s.nb * q.npw;
    DBuf<double2> tmpd;
    tmpd.alloc(n);
    CK(cudaMemcpyAsync(tmpd.p, raw, n * sizeof(double2), cudaMemcpyHostToDevice, st));
    convert_in(tmpd.p, q.X.p, n);
    launch_shape_init<T>(q.X.p, q.npw, q.kin_d.p, s.nb, q.npw, st);
    orthonormalize(s, q, s.nb);
    CK(cudaStreamSynchronize(st));
    q.have_orbitals = true;
    q.have_eig = false;
  }
  // X <- X L^{-H} with X^H S_I X = L L^H (Cholesky-QR in the metric of the subsystem's overlap)
  void orthonormalize(Sub<T>& sb, KP<T>& q, int nb) {
    ensure_small(nb);
    V2.ensure((size_t)nb * q.npw);
    gwork.ensure(gemm_hn_work(nb, nb, q.npw));
    if (sb.uspp) {
      apply_s(sb, q, q.X.p, V2.p, nb);
      launch_gemm_hn<T>(q.X.p, q.npw, V2.p, q.npw, nb, nb, q.npw, S.p, nb, gwork.p, st);
    } else {
      launch_gemm_hn<T>(q.X.p, q.npw, q.X.p, q.npw, nb, nb, q.npw, S.p, nb, gwork.p, st);
    }
    launch_hermitize(S.p, nb, st);
    launch_cholesky_inv(S.p, nb, L.p, Li.p, status.p, rel_pivot(), st);
    check_cholesky();
    // U[i][j] = conj(Li[j][i])
    launch_small_gemm(Li.p, nb, 1, identity(nb), nb, 0, nb, nb, nb, Cc.p, nb, st);
    launch_gemm_rot<T>(q.X.p, q.npw, Cc.p, nb, nb, nb, q.npw, V2.p, q.npw, 1.0, 0.0, st);
    CK(cudaMemcpyAsync(q.X.p, V2.p, (size_t)nb * q.npw * sizeof(C), cudaMemcpyDeviceToDevice, st));
  }
  DBuf<double2> eye;
  int eye_n = 0;
  const double2* identity(int n) {
    if (eye_n != n) {
      std::vector<double2> h((size_t)n * n, make_double2(0, 0));
      for (int i = 0; i < n; ++i) h[(size_t)i * n + i] = make_double2(1, 0);
      eye.alloc(h.size());
      CK(cudaMemcpy(eye.p, h.data(), h.size() * sizeof(double2), cudaMemcpyHostToDevice));
      eye_n = n;
    }
    REQ(eye_n == n, FDE_EINVAL, "identity size");
    return eye.p;
  }
  // Smallest accepted Cholesky pivot of a Gram matrix relative to its diagonal.  A pivot is the
  // squared norm of a direction's part outside the earlier ones, and it carries the Gram
  // matrix's absolute rounding error, ~1e-6 of the diagonal for FP32 vectors (split-TF32
  // products): a pivot within ten times that error counts as a dependent direction (the
  // previous directions are dropped first, then the iteration ends with the current orbitals).
  // A stricter bound (1e-3) ends the FP32 solves of the 72 x 72 x 180 slab after a dozen
  // iterations, short of a 1e-4 residual.  FP64 vectors: a rounding-level bound.
  static constexpr double rel_pivot() { return sizeof(T) == 4 ? 1e-5 : 1e-29; }
  void check_cholesky() {
    unsigned h = 0;
    CK(cudaMemcpyAsync(&h, status.p, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (h & ST_CHOLESKY) {
      CK(cudaMemsetAsync(status.p, 0, sizeof(unsigned), st));
      throw Err{FDE_ENOCONV, "overlap matrix is not positive definite (linearly dependent vectors)"};
    }
  }
  void ensure_small(int n) {
    const size_t n2 = (size_t)n * n;
    S.ensure(n2); Hs.ensure(n2); L.ensure(n2); Li.ensure(n2); Ht.ensure(n2); Y.ensure(n2); Cc.ensure(n2);
    tmp.ensure(n2); jwork.ensure(n2);
    wv.ensure(n); dnorm.ensure(n); deps.ensure(n); dtb.ensure(n); didx.ensure(n);
  }

  void set_orbitals(int i, int k, const double* d_psi) override {
    REQ(d_psi, FDE_EINVAL, "null orbitals");
    Sub<T>& s = sub(i);
    KP<T>& q = kpt(i, k);
    convert_in((const double2*)d_psi, q.X.p, (size_t)s.nb * q.npw);
    q.have_orbitals = true;
    q.have_eig = false;
  }
  void get_hpsi(int i, int k, double* d_hpsi) override {
    REQ(d_hpsi, FDE_EINVAL, "null output");
    Sub<T>& s = sub(i);
    KP<T>& q = kpt(i, k);
    convert_out(q.HX.p, (double2*)d_hpsi, (size_t)s.nb * q.npw);
    CK(cudaStreamSynchronize(st));
  }
  void get_orbitals(int i, int k, double* d_psi, double* eig, double* occ) override {
    Sub<T>& s = sub(i);
    KP<T>& q = kpt(i, k);
    if (d_psi) convert_out(q.X.p, (double2*)d_psi, (size_t)s.nb * q.npw);
    if (eig) memcpy(eig, q.eig.data(), s.nb * sizeof(double));
    if (occ) memcpy(occ, q.occ.data(), s.nb * sizeof(double));
    CK(cudaStreamSynchronize(st));
  }

  // ---- Rayleigh-Ritz on the n rows of V / HV; keeps the lowest nb pairs in V2 / HV2 ------------
  // The coefficients of the kept pairs stay in Cc ([n][n], column j = pair j).
  // With use_s (ultrasoft-like subsystems) the rows of SV are the S-images of V: the subspace
  // overlap is V^H S V and the kept S-images are rotated into SV2 alongside.
  bool use_s = false;
  DBuf<C> SV, SV2, SPb;
  void rayleigh_ritz(KP<T>& q, int n, int nb, std::vector<double>& eps) {
    const int K = q.npw;
    gwork.ensure(gemm_hn_work(n, n, K));
    launch_gemm_hn<T>(V.p, K, use_s ? SV.p : V.p, K, n, n, K, S.p, n, gwork.p, st);
    launch_gemm_hn<T>(V.p, K, HV.p, K, n, n, K, Hs.p, n, gwork.p, st);
    launch_hermitize(S.p, n, st);
    launch_hermitize(Hs.p, n, st);
    launch_cholesky_inv(S.p, n, L.p, Li.p, status.p, rel_pivot(), st);
    check_cholesky();
    launch_small_gemm(Li.p, n, 0, Hs.p, n, 0, n, n, n, tmp.p, n, st);
    launch_small_gemm(tmp.p, n, 0, Li.p, n, 1, n, n, n, Ht.p, n, st);
    launch_hermitize(Ht.p, n, st);
    hwork.ensure(heev_work_doubles(n, nb));
    launch_heev(Ht.p, n, nb, wv.p, Y.p, hwork.p, st);
    launch_small_gemm(Li.p, n, 1, Y.p, n, 0, n, n, n, Cc.p, n, st);
    launch_gemm_rot<T>(V.p, K, Cc.p, n, n, nb, K, V2.p, K, 1.0, 0.0, st);
    launch_gemm_rot<T>(HV.p, K, Cc.p, n, n, nb, K, HV2.p, K, 1.0, 0.0, st);
    if (use_s) launch_gemm_rot<T>(SV.p, K, Cc.p, n, n, nb, K, SV2.p, K, 1.0, 0.0, st);
    eps.resize(n);
    CK(cudaMemcpyAsync(eps.data(), wv.p, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    eps.resize(nb);
  }

  // Orthogonalise the m rows B against the nb current orbitals (rows 0..nb of V; in the S
  // metric, with their S-images in SV, when use_s), apply the same change to their H-images HB
  // and S-images SB when given, and normalise the rows (HB, SB alike).
  void orth_block(KP<T>& q, int nb, C* Bk, C* HBk, int m, C* SBk = nullptr) {
    const int K = q.npw;
    gwork.ensure(gemm_hn_work(nb, m, K));
    launch_gemm_hn<T>(use_s ? SV.p : V.p, K, Bk, K, nb, m, K, Cc.p, m, gwork.p, st);
    launch_gemm_rot<T>(V.p, K, Cc.p, m, nb, m, K, Bk, K, -1.0, 1.0, st);
    if (HBk) launch_gemm_rot<T>(HV.p, K, Cc.p, m, nb, m, K, HBk, K, -1.0, 1.0, st);
    if (SBk) launch_gemm_rot<T>(SV.p, K, Cc.p, m, nb, m, K, SBk, K, -1.0, 1.0, st);
    std::vector<double> sc(m);
    launch_row_norms<T>(Bk, K, m, K, nullptr, dnorm.p, nullptr, st);
    CK(cudaMemcpyAsync(sc.data(), dnorm.p, m * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int a = 0; a < m; ++a) sc[a] = 1.0 / sqrt(std::max(sc[a], 1e-300));
    CK(cudaMemcpyAsync(dtb.p, sc.data(), m * sizeof(double), cudaMemcpyHostToDevice, st));
    launch_scale_rows<T>(Bk, K, m, K, dtb.p, st);
    if (HBk) launch_scale_rows<T>(HBk, K, m, K, dtb.p, st);
    if (SBk) launch_scale_rows<T>(SBk, K, m, K, dtb.p, st);
  }

  // Block eigensolver (LOBPCG form of block Davidson): the search space of every iteration is
  // the current orbitals X, the TPA-preconditioned residuals W of the unconverged bands and
  // their previous update directions P; Rayleigh-Ritz in FP64 keeps the lowest nb pairs.
  fde_status subspace_solve(int i, int k, double tol, int max_iter, int* iters, int precond) override {
    const bool learned = precond == FDE_PRECOND_LEARNED;
    if (learned) REQ(have_pw, FDE_EINVAL, "learned preconditioner has no weights");
    bool fallback = false;  // TPA takes over when the residual stalls
    double best = 1e300;
    int stalls = 0;
    Sub<T>& s = sub(i);
    KP<T>& q = kpt(i, k);
    REQ(q.have_orbitals, FDE_EINVAL, "orbitals of this (subsystem, k) are not set");
    const int nb = s.nb, K = q.npw;
    const size_t rowsz = (size_t)K * sizeof(C);
    V.ensure((size_t)3 * nb * K);
    HV.ensure((size_t)3 * nb * K);
    V2.ensure((size_t)nb * K);
    HV2.ensure((size_t)nb * K);
    R.ensure((size_t)nb * K);
    Pb.ensure((size_t)nb * K);
    HPb.ensure((size_t)nb * K);
    ensure_small(3 * nb);
    // ultrasoft-like subsystems solve H psi = e S psi: every search vector carries its S-image
    use_s = s.uspp;
    if (use_s) {
      // the learned preconditioner is trained on norm-conserving residuals: the kinetic one
      // serves ultrasoft-like subsystems, and their iterates are not recorded
      fallback = true;
      SV.ensure((size_t)3 * nb * K);
      SV2.ensure((size_t)nb * K);
      SPb.ensure((size_t)nb * K);
    }
    std::vector<double> eps;
    CK(cudaMemcpyAsync(V.p, q.X.p, nb * rowsz, cudaMemcpyDeviceToDevice, st));
    apply_h_dev(s, q, V.p, HV.p, nb);
    if (use_s) apply_s(s, q, V.p, SV.p, nb);
    rayleigh_ritz(q, nb, nb, eps);
    CK(cudaMemcpyAsync(V.p, V2.p, nb * rowsz, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(HV.p, HV2.p, nb * rowsz, cudaMemcpyDeviceToDevice, st));
    if (use_s) CK(cudaMemcpyAsync(SV.p, SV2.p, nb * rowsz, cudaMemcpyDeviceToDevice, st));
    int it = 0;
    bool conv = false, havep = false;
    std::vector<double> rn(nb), tb(nb);
    for (;;) {
      CK(cudaMemcpyAsync(deps.p, eps.data(), nb * sizeof(double), cudaMemcpyHostToDevice, st));
      launch_residual<T>(HV.p, use_s ? SV.p : V.p, deps.p, nb, K, K, R.p, K, st);  // R = H psi - e S psi
      launch_row_norms<T>(R.p, K, nb, K, nullptr, dnorm.p, nullptr, st);
      CK(cudaMemcpyAsync(rn.data(), dnorm.p, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      std::vector<int> sel;
      for (int j = 0; j < nb; ++j) {
        REQ(std::isfinite(rn[j]), FDE_ENONFINITE, "non-finite residual");
        if (sqrt(rn[j]) >= tol) sel.push_back(j);
      }
      if (sel.empty()) { conv = true; break; }
      if (it >= max_iter) break;
      if (it < precond_record && !use_s) {
        // keep (R, X) of this iterate; the correction target (1 - P) X is formed once the
        // converged block P is known
        auto p = std::make_unique<Pairs>();
        p->sub = i;
        p->k = k;
        p->n = nb;
        p->R.alloc((size_t)nb * K);
        p->D.alloc((size_t)nb * K);
        p->tb.alloc(nb);
        CK(cudaMemcpyAsync(p->R.p, R.p, nb * rowsz, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(p->D.p, V.p, nb * rowsz, cudaMemcpyDeviceToDevice, st));
        launch_row_norms<T>(V.p, K, nb, K, q.kin_d.p, p->tb.p, nullptr, st);
        recorded.push_back(std::move(p));
      }
      ++it;
      const int m = (int)sel.size();
      CK(cudaMemcpyAsync(didx.p, sel.data(), m * sizeof(int), cudaMemcpyHostToDevice, st));
      C* W = V.p + (size_t)nb * K;
      launch_gather_rows<T>(R.p, K, didx.p, m, K, W, K, st);
      launch_row_norms<T>(V.p, K, nb, K, q.kin_d.p, dnorm.p, nullptr, st);
      CK(cudaMemcpyAsync(tb.data(), dnorm.p, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      std::vector<double> tsel(m);
      for (int a = 0; a < m; ++a) tsel[a] = tb[sel[a]];
      CK(cudaMemcpyAsync(dtb.p, tsel.data(), m * sizeof(double), cudaMemcpyHostToDevice, st));
      if (learned && !fallback) {
        double worst = 0;
        std::vector<double> ss(m);
        for (int a = 0; a < m; ++a) {
          ss[a] = rn[sel[a]];
          worst = std::max(worst, rn[sel[a]]);
        }
        // stall test: three iterations without a 1% drop of the largest residual
        if (worst > 0.99 * best) {
          if (++stalls >= 3) fallback = true;
        } else {
          stalls = 0;
        }
        best = std::min(best, worst);
        dss.ensure(m);
        CK(cudaMemcpyAsync(dss.p, ss.data(), m * sizeof(double), cudaMemcpyHostToDevice, st));
      }
      if (learned && !fallback)
        launch_precond_apply<T>(W, K, q.kin_d.p, dtb.p, dss.p, m, K, pwb.p, W, K, st);
      else
        launch_tpa<T>(W, K, q.kin_d.p, dtb.p, m, K, W, K, st);
      orth_block(q, nb, W, nullptr, m);
      int np = 0;
      if (havep) {
        C* P = V.p + (size_t)(nb + m) * K;
        C* HP = HV.p + (size_t)(nb + m) * K;
        C* SP = use_s ? SV.p + (size_t)(nb + m) * K : nullptr;
        launch_gather_rows<T>(Pb.p, K, didx.p, m, K, P, K, st);
        launch_gather_rows<T>(HPb.p, K, didx.p, m, K, HP, K, st);
        if (use_s) launch_gather_rows<T>(SPb.p, K, didx.p, m, K, SP, K, st);
        orth_block(q, nb, P, HP, m, SP);
        np = m;
      }
      apply_h_dev(s, q, W, HV.p + (size_t)nb * K, m);
      if (use_s) apply_s(s, q, W, SV.p + (size_t)nb * K, m);
      int n = nb + m + np;
      try {
        rayleigh_ritz(q, n, nb, eps);
      } catch (Err& e) {
        if (e.st != FDE_ENOCONV) throw;
        if (np == 0) break;  // dependent search directions: keep the current orbitals
        n = nb + m;          // drop the previous directions and retry once
        try {
          rayleigh_ritz(q, n, nb, eps);
        } catch (Err& e2) {
          if (e2.st != FDE_ENOCONV) throw;
          break;
        }
      }
      // update directions P = [W P] C[nb:n, :nb] (and their H- and S-images)
      launch_gemm_rot<T>(V.p + (size_t)nb * K, K, Cc.p + (size_t)nb * n, n, n - nb, nb, K, Pb.p, K, 1.0, 0.0, st);
      launch_gemm_rot<T>(HV.p + (size_t)nb * K, K, Cc.p + (size_t)nb * n, n, n - nb, nb, K, HPb.p, K, 1.0, 0.0, st);
      if (use_s)
        launch_gemm_rot<T>(SV.p + (size_t)nb * K, K, Cc.p + (size_t)nb * n, n, n - nb, nb, K, SPb.p, K, 1.0, 0.0, st);
      CK(cudaMemcpyAsync(V.p, V2.p, nb * rowsz, cudaMemcpyDeviceToDevice, st));
      CK(cudaMemcpyAsync(HV.p, HV2.p, nb * rowsz, cudaMemcpyDeviceToDevice, st));
      if (use_s) CK(cudaMemcpyAsync(SV.p, SV2.p, nb * rowsz, cudaMemcpyDeviceToDevice, st));
      if constexpr (sizeof(T) == 4) {
        // FP32: one more Rayleigh-Ritz step on the kept block alone.  The big step's inverse
        // Cholesky factor scales the split-TF32 Gram matrix's rounding into the kept basis; its
        // own Gram matrix is near the identity, so this step re-orthonormalises it and makes
        // the Ritz values those of an orthonormal basis (without it, solves near the FP32
        // residual floor returned Ritz values below the true eigenvalues)
        // every eighth iteration the kept block's H- and S-images are recomputed rather than
        // carried: they are rotated by the inverse Cholesky factors of every step, which scale
        // their FP32 rounding up, and a drifted image shifts the Ritz values
        if (it % 8 == 0) {
          apply_h_dev(s, q, V.p, HV.p, nb);
          if (use_s) apply_s(s, q, V.p, SV.p, nb);
        }
        try {
          rayleigh_ritz(q, nb, nb, eps);
          CK(cudaMemcpyAsync(V.p, V2.p, nb * rowsz, cudaMemcpyDeviceToDevice, st));
          CK(cudaMemcpyAsync(HV.p, HV2.p, nb * rowsz, cudaMemcpyDeviceToDevice, st));
          if (use_s) CK(cudaMemcpyAsync(SV.p, SV2.p, nb * rowsz, cudaMemcpyDeviceToDevice, st));
        } catch (Err& e) {
          if (e.st != FDE_ENOCONV) throw;
        }
      }
      havep = true;
    }
    if (conv) {
      // recorded iterates: D = (1 - P) X with P the projector on the converged block (rows of V)
      for (auto& p : recorded) {
        gwork.ensure(gemm_hn_work(nb, nb, K));
        launch_gemm_hn<T>(V.p, K, p->D.p, K, nb, nb, K, Cc.p, nb, gwork.p, st);
        launch_gemm_rot<T>(V.p, K, Cc.p, nb, nb, nb, K, p->D.p, K, -1.0, 1.0, st);
        pair_stats(*p, q);
        CK(cudaStreamSynchronize(st));
        pairs.push_back(std::move(p));
      }
    }
    recorded.clear();
    CK(cudaMemcpyAsync(q.X.p, V.p, nb * rowsz, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(q.HX.p, HV.p, nb * rowsz, cudaMemcpyDeviceToDevice, st));
    q.eig = eps;
    q.have_eig = true;
    CK(cudaStreamSynchronize(st));
    if (iters) *iters = it;
    return conv ? FDE_OK : FDE_ENOCONV;
  }

  // ---- occupations and density ----------------------------------------------------------------
  void occupations(Sub<T>& s) {
    std::vector<double> eig((size_t)s.nk * s.nb), occ((size_t)s.nk * s.nb);
    for (int k = 0; k < s.nk; ++k) std::copy(s.kp[k].eig.begin(), s.kp[k].eig.end(), eig.begin() + (size_t)k * s.nb);
    double mu = 0, ts = 0;
    REQ(occupations_host(s.nk, s.nb, eig.data(), s.wk.data(), s.nelec, s.smearing, occ.data(), &mu, &ts,
                         s.smear_kind),
        FDE_EINVAL, "inconsistent occupation arguments");
    for (int k = 0; k < s.nk; ++k) s.kp[k].occ.assign(occ.begin() + (size_t)k * s.nb, occ.begin() + (size_t)(k + 1) * s.nb);
    s.mu = mu;
    s.entropy = ts;
  }

  void density_from_orbitals(Sub<T>& s, double* out) {
    occw.ensure(s.nb);
    for (int k = 0; k < s.nk; ++k) {
      KP<T>& q = s.kp[k];
      std::vector<double> w(s.nb);
      for (int j = 0; j < s.nb; ++j) w[j] = 2.0 * s.wk[k] * q.occ[j] / omega;
      CK(cudaMemcpyAsync(occw.p, w.data(), s.nb * sizeof(double), cudaMemcpyHostToDevice, st));
      scratch.ensure((size_t)s.nb * g.n3 * q.sp.ncol);
      launch_density<T>(q.X.p, q.npw, s.nb, occw.p, scratch.p, rho_plane.p, k > 0, q.sp, g, plans.fp, st);
      CK(cudaStreamSynchronize(st));  // occw is reused by the next k
    }
    launch_transpose<double, double>(rho_plane.p, out, g.n3, (int)((long long)g.n1 * g.n2), 0, st);
    if (s.uspp) augment_density(s, out);
    if (sym.n > 1) {  // densities from an irreducible k-set: average over the symmetry group
      grid_symmetrize(out, rho_plane.p, g, sym, st);
      CK(cudaMemcpyAsync(out, rho_plane.p, nr * sizeof(double), cudaMemcpyDeviceToDevice, st));
    }
    grid_nonfinite(out, nr, status.p, st);
  }

  // Augmentation charges of an ultrasoft-like subsystem added to its density:
  // rho += sum_a g_a(r) c_a, c_a = sum_ij q_ij 2 sum_k w_k sum_j n_jk Re <u_jk|beta_ai><beta_aj|u_jk>,
  // so that int rho_I = N_I for S-normalised orbitals.  The projections come to the host (a
  // natoms x nproj x nb block per k), the charges are placed in reciprocal space and transformed.
  void augment_density(Sub<T>& s, double* out) {
    std::vector<double> ca(s.natoms, 0.0);
    const int np = s.nproj_atom;
    for (int k = 0; k < s.nk; ++k) {
      KP<T>& q = s.kp[k];
      gwork.ensure(gemm_hn_work(s.nproj, s.nb, q.npw));
      Pm.ensure((size_t)s.nproj * s.nb);
      launch_gemm_hn<T>(q.beta.p, q.npw, q.X.p, q.npw, s.nproj, s.nb, q.npw, Pm.p, s.nb, gwork.p, st);
      std::vector<double2> P((size_t)s.nproj * s.nb);
      CK(cudaMemcpyAsync(P.data(), Pm.p, P.size() * sizeof(double2), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      for (int a = 0; a < s.natoms; ++a)
        for (int i = 0; i < np; ++i)
          for (int i2 = 0; i2 < np; ++i2) {
            double b = 0;
            for (int j = 0; j < s.nb; ++j) {
              const double2 x = P[(size_t)(a * np + i) * s.nb + j], y = P[(size_t)(a * np + i2) * s.nb + j];
              b += q.occ[j] * (x.x * y.x + x.y * y.y);
            }
            ca[a] += 2.0 * s.wk[k] * s.Q[i * np + i2] * b;
          }
    }
    DBuf<double> dc;
    dc.alloc(s.natoms);
    CK(cudaMemcpyAsync(dc.p, ca.data(), s.natoms * sizeof(double), cudaMemcpyHostToDevice, st));
    double2* A = cb[0].p;
    grid_aug_density_g(A, g, cell, s.aug_pos.p, dc.p, s.natoms, s.aug_sigma, st);
    launch_fft3d<double>(A, g, plans64.fp, +1, st);
    grid_combine<double>(out, nullptr, nullptr, A, 1.0, out, nr, st);
    CK(cudaStreamSynchronize(st));  // dc is released on return
  }

  // Point-group operations the densities are symmetrised over (sign flips about the origin).
  // They must form a group and map every subsystem's atoms onto atoms of the same subsystem
  // and charge: then each H_I commutes with them and a density built from an irreducible set
  // of k-points becomes the full-mesh density once averaged over the group.
  SymOps sym{1, {0, 0, 0, 0, 0, 0, 0, 0}};
  void set_symmetry(int nops, const int* ops) override {
    REQ(nops >= 1 && nops <= 8 && ops, FDE_EINVAL, "between 1 and 8 operations");
    std::vector<int> m(ops, ops + nops);
    std::sort(m.begin(), m.end());
    REQ(m[0] == 0, FDE_EINVAL, "the identity (mask 0) must be one of the operations");
    for (int a : m) {
      REQ(a >= 0 && a <= 7, FDE_EINVAL, "operation masks are 3-bit sign flips");
      for (int b : m) REQ(std::binary_search(m.begin(), m.end(), a ^ b), FDE_EINVAL, "the operations must form a group");
    }
    REQ(std::adjacent_find(m.begin(), m.end()) == m.end(), FDE_EINVAL, "repeated operation");
    const double Lc[3] = {A[0][0], A[1][1], A[2][2]};
    for (auto& sp : subs) {
      std::vector<int> have;
      symmetry_ops_host(Lc, sp->natoms, sp->pos.data(), sp->Z.data(), 1e-6, have);
      for (int a : m)
        REQ(std::find(have.begin(), have.end(), a) != have.end(), FDE_EINVAL,
            "an operation does not map a subsystem's atoms onto themselves");
    }
    sym.n = nops;
    for (int i = 0; i < 8; ++i) sym.mask[i] = i < nops ? m[i] : 0;
  }

  void update_density(int i) override {
    Sub<T>& s = sub(i);
    for (auto& q : s.kp) REQ(q.have_eig, FDE_EINVAL, "eigenvalues not available: run fde_subspace_solve first");
    occupations(s);
    density_from_orbitals(s, s.rho.p);
    sync();
  }

  // ---- energies ---------------------------------------------------------------------------------
  // Janak kinetic and nonlocal energies of one subsystem's stored orbitals.
  void band_terms(Sub<T>& s, double* T_J, double* E_nl) {
    *T_J = 0;
    *E_nl = 0;
    std::vector<double> t(s.nb);
    for (int k = 0; k < s.nk; ++k) {
      KP<T>& q = s.kp[k];
      if (!q.have_orbitals) continue;
      dnorm.ensure(s.nb);
      launch_row_norms<T>(q.X.p, q.npw, s.nb, q.npw, q.kin_d.p, dnorm.p, nullptr, st);
      CK(cudaMemcpyAsync(t.data(), dnorm.p, s.nb * sizeof(double), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      for (int j = 0; j < s.nb; ++j) *T_J += 2.0 * s.wk[k] * q.occ[j] * t[j];
      if (s.nproj) {
        gwork.ensure(gemm_hn_work(s.nproj, s.nb, q.npw));
        Pm.ensure((size_t)s.nproj * s.nb);
        launch_gemm_hn<T>(q.beta.p, q.npw, q.X.p, q.npw, s.nproj, s.nb, q.npw, Pm.p, s.nb, gwork.p, st);
        std::vector<double2> P((size_t)s.nproj * s.nb);
        CK(cudaMemcpyAsync(P.data(), Pm.p, P.size() * sizeof(double2), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        for (int j = 0; j < s.nb; ++j) {
          double e = 0;
          for (int a = 0; a < s.natoms; ++a)
            for (int p1 = 0; p1 < s.nproj_atom; ++p1)
              for (int p2 = 0; p2 < s.nproj_atom; ++p2) {
                const double2 x = P[(size_t)(a * s.nproj_atom + p1) * s.nb + j];
                const double2 y = P[(size_t)(a * s.nproj_atom + p2) * s.nb + j];
                e += s.D[p1 * s.nproj_atom + p2] * (x.x * y.x + x.y * y.y);
              }
          *E_nl += 2.0 * s.wk[k] * q.occ[j] * e;
        }
      }
    }
  }

  double integrate_product(const double* a, const double* b, long long n = 0) {
    grid_dot_partial(a, b, n > 0 ? n : nr, 0, partial.p, st);
    grid_finalize(partial.p, 1, omega / (double)nr, scal.p + 255, st);
    double h = 0;
    CK(cudaMemcpyAsync(&h, scal.p + 255, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return h;
  }
  double integrate_absdiff(const double* a, const double* b) {
    grid_dot_partial(a, b, nr, 1, partial.p, st);
    grid_finalize(partial.p, 1, omega / (double)nr, scal.p + 255, st);
    double h = 0;
    CK(cudaMemcpyAsync(&h, scal.p + 255, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return h;
  }

  void energy(fde_energies* out) override {
    REQ(out, FDE_EINVAL, "null output");
    memset(out, 0, sizeof(*out));
    ensure_vloc();
    EnergyParts ep = grid_pass(false, true, -1);
    double TJ = 0, Enl = 0, TS = 0, band = 0, deband = 0;
    for (auto& sp : subs) {
      double t, e;
      band_terms(*sp, &t, &e);
      TJ += t;
      Enl += e;
      TS += sp->entropy;
      for (int k = 0; k < sp->nk; ++k)
        for (int j = 0; j < sp->nb; ++j) band += 2.0 * sp->wk[k] * sp->kp[k].occ[j] * sp->kp[k].eig[j];
      deband -= integrate_product(sp->veff.p, sp->rho.p);
    }
    out->E_kin = TJ;
    out->E_nl = Enl;
    out->E_loc = ep.Eloc;
    out->E_H = ep.EH;
    out->E_xc = ep.Exc;
    out->T_nad = ep.Ttot - ep.Tsub;
    out->E_xc_nad = ep.Exc - ep.Exc_sub;
    out->E_H_nad = ep.EH - ep.EH_sub;
    out->E_nn = enn;
    out->E_fde = TJ + Enl + ep.Eloc + ep.EH + ep.Exc + out->T_nad + enn;
    out->TS = TS;
    out->F_fde = out->E_fde - TS;
    out->E_band_form = band + deband + ep.Eloc + ep.EH + ep.Exc + out->T_nad + enn;
  }

  // ---- learned preconditioner ----------------------------------------------------------------
  DBuf<float> pw, pm1, pm2, pround, gpart;
  DBuf<unsigned short> pwb;
  DBuf<double> gsum, dss, awork;
  DBuf<C> gtmp;  // m R with the master weights (tensor-core training's scale pass)
  bool have_pw = false;
  int adam_step = 0;
  int precond_mode = FDE_PRECOND_TPA;
  struct Pairs {
    int sub = 0, k = 0, n = 0;
    DBuf<cplx<T>> R, D;
    DBuf<double> tb, ss, dn;
  };
  std::vector<std::unique_ptr<Pairs>> pairs;

  void ensure_pw() {
    if (pw.n) return;
    pw.alloc(kPrecondParams);
    pm1.alloc(kPrecondParams);
    pm2.alloc(kPrecondParams);
    pround.alloc(kPrecondParams);
    pwb.alloc(kPrecondParams);
    gsum.alloc(kPrecondParams + 1);
  }
  void set_precond_mode(int mode) override {
    REQ(mode == FDE_PRECOND_TPA || mode == FDE_PRECOND_LEARNED, FDE_EINVAL, "unknown preconditioner");
    if (mode == FDE_PRECOND_LEARNED) REQ(have_pw, FDE_EINVAL, "learned preconditioner has no weights");
    precond_mode = mode;
  }
  void precond_set_weights(const float* h) override {
    REQ(h, FDE_EINVAL, "null weights");
    ensure_pw();
    CK(cudaMemcpyAsync(pw.p, h, kPrecondParams * sizeof(float), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(pm1.p, 0, kPrecondParams * sizeof(float), st));
    CK(cudaMemsetAsync(pm2.p, 0, kPrecondParams * sizeof(float), st));
    launch_precond_to_bf16(pw.p, pwb.p, pround.p, st);
    CK(cudaStreamSynchronize(st));
    adam_step = 0;
    have_pw = true;
  }
  void precond_get_weights(float* h, float* hb) override {
    REQ(have_pw, FDE_EINVAL, "no weights");
    if (h) CK(cudaMemcpyAsync(h, pw.p, kPrecondParams * sizeof(float), cudaMemcpyDeviceToHost, st));
    if (hb) {
      launch_precond_to_bf16(pw.p, pwb.p, pround.p, st);
      CK(cudaMemcpyAsync(hb, pround.p, kPrecondParams * sizeof(float), cudaMemcpyDeviceToHost, st));
    }
    CK(cudaStreamSynchronize(st));
  }
  void precond_clear() override { pairs.clear(); }
  int precond_record = 0;  // record (residual, iterate) pairs of the first iterations of each solve
  std::vector<std::unique_ptr<Pairs>> recorded;
  void set_precond_record(int n) override { precond_record = std::max(0, n); }
  void stats(long long* dav, long long* hpsi) override {
    if (dav) *dav = davidson_iters;
    if (hpsi) *hpsi = hpsi_bands;
  }
  // Row statistics of a pair set: band kinetic energies come with it; |R_j|^2, |D_j|^2 here.
  void pair_stats(Pairs& p, KP<T>& q) {
    p.ss.alloc(p.n);
    p.dn.alloc(p.n);
    launch_row_norms<T>(p.R.p, q.npw, p.n, q.npw, nullptr, p.ss.p, nullptr, st);
    launch_row_norms<T>(p.D.p, q.npw, p.n, q.npw, nullptr, p.dn.p, nullptr, st);
  }
  void precond_add_pairs(int i, int k, int n, const double* r, const double* d, const double* tb) override {
    REQ(r && d && tb && n > 0, FDE_EINVAL, "bad pair arguments");
    KP<T>& q = kpt(i, k);
    auto p = std::make_unique<Pairs>();
    p->sub = i;
    p->k = k;
    p->n = n;
    const size_t cnt = (size_t)n * q.npw;
    p->R.alloc(cnt);
    p->D.alloc(cnt);
    p->tb.alloc(n);
    DBuf<double2> tmpd;
    tmpd.alloc(cnt);
    CK(cudaMemcpyAsync(tmpd.p, r, cnt * sizeof(double2), cudaMemcpyHostToDevice, st));
    convert_in(tmpd.p, p->R.p, cnt);
    CK(cudaStreamSynchronize(st));
    CK(cudaMemcpyAsync(tmpd.p, d, cnt * sizeof(double2), cudaMemcpyHostToDevice, st));
    convert_in(tmpd.p, p->D.p, cnt);
    CK(cudaMemcpyAsync(p->tb.p, tb, n * sizeof(double), cudaMemcpyHostToDevice, st));
    pair_stats(*p, q);
    CK(cudaStreamSynchronize(st));
    pairs.push_back(std::move(p));
  }
  // Training pairs from the converged orbitals of (sub, k): seeded smooth perturbations D
  // orthogonal to the converged block, R = (H - eps_j) D_j; the ideal correction of R is D.
  void precond_harvest(int i, int k, const double* raw, int n) override {
    REQ(raw && n > 0, FDE_EINVAL, "bad harvest arguments");
    Sub<T>& s = sub(i);
    KP<T>& q = kpt(i, k);
    REQ(q.have_eig, FDE_EINVAL, "harvest needs converged orbitals (run fde_subspace_solve first)");
    n = std::min(n, s.nb);
    const int K = q.npw;
    auto p = std::make_unique<Pairs>();
    p->sub = i;
    p->k = k;
    p->n = n;
    p->R.alloc((size_t)n * K);
    p->D.alloc((size_t)n * K);
    p->tb.alloc(n);
    DBuf<double2> tmpd;
    tmpd.alloc((size_t)n * K);
    CK(cudaMemcpyAsync(tmpd.p, raw, (size_t)n * K * sizeof(double2), cudaMemcpyHostToDevice, st));
    convert_in(tmpd.p, p->D.p, (size_t)n * K);
    launch_shape_init<T>(p->D.p, K, q.kin_d.p, n, K, st);
    ensure_small(std::max(3 * s.nb, n));
    gwork.ensure(gemm_hn_work(s.nb, n, K));
    launch_gemm_hn<T>(q.X.p, K, p->D.p, K, s.nb, n, K, Cc.p, n, gwork.p, st);
    launch_gemm_rot<T>(q.X.p, K, Cc.p, n, s.nb, n, K, p->D.p, K, -1.0, 1.0, st);
    std::vector<double> sc(n);
    launch_row_norms<T>(p->D.p, K, n, K, nullptr, dnorm.p, nullptr, st);
    CK(cudaMemcpyAsync(sc.data(), dnorm.p, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int a = 0; a < n; ++a) sc[a] = 1.0 / sqrt(std::max(sc[a], 1e-300));
    CK(cudaMemcpyAsync(dtb.p, sc.data(), n * sizeof(double), cudaMemcpyHostToDevice, st));
    launch_scale_rows<T>(p->D.p, K, n, K, dtb.p, st);
    apply_h_dev(s, q, p->D.p, p->R.p, n);
    CK(cudaMemcpyAsync(deps.p, q.eig.data(), n * sizeof(double), cudaMemcpyHostToDevice, st));
    launch_residual<T>(p->R.p, p->D.p, deps.p, n, K, K, p->R.p, K, st);
    launch_row_norms<T>(q.X.p, K, n, K, q.kin_d.p, p->tb.p, nullptr, st);
    pair_stats(*p, q);
    CK(cudaStreamSynchronize(st));
    pairs.push_back(std::move(p));
  }
  void precond_loss_grad(double* grad, double* loss) override {
    REQ(have_pw, FDE_EINVAL, "no weights");
    REQ(!pairs.empty(), FDE_EINVAL, "no training pairs");
    std::vector<double> acc(kPrecondParams + 1, 0.0), h(kPrecondParams + 1);
    for (auto& pp : pairs) {
      Pairs& p = *pp;
      KP<T>& q = kpt(p.sub, p.k);
      gpart.ensure((size_t)precond_grad_blocks(p.n, q.npw) * (kPrecondParams + 1));
      awork.ensure(precond_alpha_work(p.n));
      gtmp.ensure((size_t)p.n * q.npw);
      launch_precond_grad<T>(p.R.p, p.D.p, p.n, q.npw, q.kin_d.p, p.tb.p, p.ss.p, p.dn.p, pw.p, gpart.p, awork.p,
                             gtmp.p, gsum.p, st);
      CK(cudaMemcpyAsync(h.data(), gsum.p, (kPrecondParams + 1) * sizeof(double), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      for (int a = 0; a <= kPrecondParams; ++a) acc[a] += h[a];
    }
    if (grad) memcpy(grad, acc.data(), kPrecondParams * sizeof(double));
    if (loss) *loss = acc[kPrecondParams];
    CK(cudaMemcpyAsync(gsum.p, acc.data(), (kPrecondParams + 1) * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
  }
  void precond_train(int steps, double lr, double* l0, double* l1) override {
    REQ(steps > 0 && lr > 0, FDE_EINVAL, "bad training arguments");
    double loss = 0;
    for (int s = 0; s < steps; ++s) {
      precond_loss_grad(nullptr, &loss);
      if (s == 0 && l0) *l0 = loss;
      launch_precond_adam(pw.p, pwb.p, gsum.p, pm1.p, pm2.p, (float)lr, ++adam_step, st);
    }
    precond_loss_grad(nullptr, &loss);
    if (l1) *l1 = loss;
  }
  void precond_apply(int i, int k, const void* r, void* w, int nb, const double* tband) override {
    REQ(r && w && tband && nb > 0, FDE_EINVAL, "bad arguments");
    REQ(have_pw, FDE_EINVAL, "no weights");
    KP<T>& q = kpt(i, k);
    DBuf<double> tb, ss;
    tb.alloc(nb);
    ss.alloc(nb);
    CK(cudaMemcpyAsync(tb.p, tband, nb * sizeof(double), cudaMemcpyHostToDevice, st));
    launch_row_norms<T>((const C*)r, q.npw, nb, q.npw, nullptr, ss.p, nullptr, st);
    launch_precond_apply<T>((const C*)r, q.npw, q.kin_d.p, tb.p, ss.p, nb, q.npw, pwb.p, (C*)w, q.npw, st);
    sync();
  }

  // ---- Pulay mixing -----------------------------------------------------------------------------
  void pulay_reset(PulayHist& h) { h.len = 0; h.head = 0; }
  void pulay_reset() { pulay_reset(hist); }
  void pulay(double* rin, const double* rout) { pulay(hist, rin, rout, nr); }
  // rho_in <- DIIS mix of the history extended by (rho_in, rho_out - rho_in); the vectors
  // hold n values (one grid, or the stacked grids of every subsystem)
  void pulay(PulayHist& hs, double* rin, const double* rout, long long n) {
    const int H = 8;
    const double beta = 0.3;
    if (hs.in.size() < (size_t)H) {
      hs.in.resize(H);
      hs.res.resize(H);
    }
    for (int h = 0; h < H; ++h) { hs.in[h].ensure(n); hs.res[h].ensure(n); }
    const int slot = (hs.head + hs.len) % H;
    if (hs.len == H) hs.head = (hs.head + 1) % H; else ++hs.len;
    CK(cudaMemcpyAsync(hs.in[slot].p, rin, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    // res = rout - rin
    CK(cudaMemcpyAsync(hs.res[slot].p, rout, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    grid_axpy(hs.res[slot].p, rin, -1.0, n, st);
    const int m = hs.len;
    std::vector<int> sl(m);
    for (int a = 0; a < m; ++a) sl[a] = (hs.head + a) % H;
    std::vector<double> ov((size_t)m * m, 0.0);
    for (int a = 0; a < m; ++a)
      for (int c = a; c < m; ++c) {
        const double v = integrate_product(hs.res[sl[a]].p, hs.res[sl[c]].p, n) * (double)nr / omega;
        ov[a * m + c] = ov[c * m + a] = v;
      }
    std::vector<double> coef(m, 0.0);
    pulay_coefficients(ov.data(), m, coef.data());
    std::vector<const double*> pi(m), pr(m);
    for (int a = 0; a < m; ++a) { pi[a] = hs.in[sl[a]].p; pr[a] = hs.res[sl[a]].p; }
    dptrs.ensure(2 * m);
    dcoef.ensure(m);
    CK(cudaMemcpyAsync(dptrs.p, pi.data(), m * sizeof(double*), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(dptrs.p + m, pr.data(), m * sizeof(double*), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(dcoef.p, coef.data(), m * sizeof(double), cudaMemcpyHostToDevice, st));
    grid_lincomb(dptrs.p, dptrs.p + m, dcoef.p, m, beta, n, rin, st);
    CK(cudaStreamSynchronize(st));
  }
  // ---- subsystem SCF and freeze-and-thaw ------------------------------------------------------
  // Inner-iteration thresholds.  One freeze-and-thaw cycle evaluates the energy with every
  // density refreshed, which is not stationary in the inner-SCF densities, so the density
  // residual int|rho_out - rho_in| is converged to 10 x the energy tolerance (FP32 orbitals
  // floor it near 1e-4 in the mixed path).
  double davidson_tol(double tol) const { return sizeof(T) == 8 ? std::max(1e-10, std::min(1e-6, tol)) : 3e-5; }
  double dres_tol(double tol) const { return sizeof(T) == 8 ? 10.0 * tol : std::max(10.0 * tol, 1e-4); }

  fde_status scf_subsystem(int I, double tol, int max_scf, fde_energies* out) override {
    Sub<T>& s = sub(I);
    for (auto& q : s.kp) REQ(q.have_orbitals, FDE_EINVAL, "orbitals of the subsystem are not set");
    ensure_vloc();
    rho_in.ensure(nr);
    CK(cudaMemcpyAsync(rho_in.p, s.rho.p, nr * sizeof(double), cudaMemcpyDeviceToDevice, st));
    // frozen band terms of the other subsystems
    double TJo = 0, Enlo = 0, TSo = 0;
    for (size_t J = 0; J < subs.size(); ++J) {
      if ((int)J == I) continue;
      double t, e;
      band_terms(*subs[J], &t, &e);
      TJo += t;
      Enlo += e;
      TSo += subs[J]->entropy;
    }
    pulay_reset();
    double Eprev = 0;
    bool have_prev = false;
    const double dtol = davidson_tol(tol);
    // Early SCF iterations need only rough eigenvectors: the eigensolver tolerance follows
    // the density residual of the previous iteration down to dtol.  An orbital error of
    // |r_j| / gap moves int|rho_out| by up to ~4 n_occ |r_j| / gap, so the residual norm is
    // held to 1e-4 x the density residual; with a looser coupling (1e-2) a small molecule's
    // eigensolver returned without iterating while its input density still moved, and the
    // Pulay iteration stalled near 1e-5.
    double dres_prev = 1.0;
    fde_energies en{};
    for (int it = 1; it <= max_scf; ++it) {
      CK(cudaMemcpyAsync(s.rho.p, rho_in.p, nr * sizeof(double), cudaMemcpyDeviceToDevice, st));
      grid_pass(true, false, I);
      for (int k = 0; k < s.nk; ++k) {
        int its = 0;
        subspace_solve(I, k, std::max(dtol, std::min(1e-3, 1e-4 * dres_prev)), 60, &its, precond_mode);
        davidson_iters += its;
      }
      occupations(s);
      density_from_orbitals(s, s.rho.p);
      sync();
      // energy of the output density with the others frozen
      EnergyParts ep = grid_pass(false, true, -1);
      double t, e;
      band_terms(s, &t, &e);
      en.E_kin = TJo + t;
      en.E_nl = Enlo + e;
      en.E_loc = ep.Eloc;
      en.E_H = ep.EH;
      en.E_xc = ep.Exc;
      en.T_nad = ep.Ttot - ep.Tsub;
      en.E_xc_nad = ep.Exc - ep.Exc_sub;
      en.E_H_nad = ep.EH - ep.EH_sub;
      en.E_nn = enn;
      en.E_fde = en.E_kin + en.E_nl + en.E_loc + en.E_H + en.E_xc + en.T_nad + enn;
      en.TS = TSo + s.entropy;
      en.F_fde = en.E_fde - en.TS;
      en.iters = it;
      const double dres = integrate_absdiff(s.rho.p, rho_in.p);
      dres_prev = dres;
      en.dE = have_prev ? en.F_fde - Eprev : 0.0;
      REQ(std::isfinite(en.F_fde), FDE_ENONFINITE, "non-finite energy");
      if (trace_level() > 0)
        fprintf(stderr, "[fde] scf sub %d it %d F %.12f dE %.3e drho %.3e eig_iters %lld\n", I, it, en.F_fde, en.dE,
                dres, davidson_iters);
      if (have_prev && fabs(en.dE) < tol && dres < dres_tol(tol)) {
        if (out) *out = en;
        return FDE_OK;
      }
      Eprev = en.F_fde;
      have_prev = true;
      pulay(rho_in.p, s.rho.p);
    }
    if (out) *out = en;
    return FDE_ENOCONV;
  }

  // One Jacobi cycle against the current densities (frozen at the cycle start).  start
  // (device [nsub][N_r], nullable): densities each subsystem SCF starts from instead of
  // its frozen one (a warm start that leaves the cycle's fixed point unchanged).
  fde_status freeze_thaw(double tol, int max_scf, fde_energies* out, const double* start) override {
    REQ(!subs.empty(), FDE_EINVAL, "no subsystems");
    ensure_vloc();
    const size_t ns = subs.size();
    frozen.ensure(ns * nr);
    fresh.ensure(ns * nr);
    for (size_t I = 0; I < ns; ++I)
      CK(cudaMemcpyAsync(frozen.p + I * nr, subs[I]->rho.p, nr * sizeof(double), cudaMemcpyDeviceToDevice, st));
    fde_status worst = FDE_OK;
    int iters = 0;
    for (size_t I = 0; I < ns; ++I) {
      for (size_t J = 0; J < ns; ++J)
        CK(cudaMemcpyAsync(subs[J]->rho.p, (start && J == I ? start : frozen.p) + J * nr, nr * sizeof(double),
                           cudaMemcpyDeviceToDevice, st));
      fde_energies e{};
      const fde_status r = scf_subsystem((int)I, tol, max_scf, &e);
      if (r != FDE_OK) worst = r;
      iters += e.iters;
      CK(cudaMemcpyAsync(fresh.p + I * nr, subs[I]->rho.p, nr * sizeof(double), cudaMemcpyDeviceToDevice, st));
    }
    for (size_t I = 0; I < ns; ++I)
      CK(cudaMemcpyAsync(subs[I]->rho.p, fresh.p + I * nr, nr * sizeof(double), cudaMemcpyDeviceToDevice, st));
    // potentials of the refreshed densities, then every energy term
    grid_pass(true, false, -1);
    if (out) {
      energy(out);
      out->iters = iters;
    }
    sync();
    return worst;
  }

  // SCF of every subsystem with the total density refreshed after every step (the paper's
  // default: the subsystem SCF of Fig. 1b runs once per exchange of the densities).  Each
  // step: V_eff^I of every subsystem from the current input densities, eigensolves of every
  // (subsystem, k), occupations and output densities, then one Pulay (DIIS) step on the
  // stacked densities of all subsystems (one set of coefficients for every subsystem: they are
  // coupled through the shared potential).  Converged when the FDE free energy changes by less than tol and every subsystem's
  // int|rho_out - rho_in| is below 10 tol (mixed precision: max(10 tol, 1e-4)).  The
  // subsystem densities hold the last output densities on return; out gets their energies.
  fde_status scf_refresh(double tol, int max_scf, fde_energies* out) override {
    REQ(!subs.empty(), FDE_EINVAL, "no subsystems");
    REQ(max_scf > 0 && tol > 0, FDE_EINVAL, "bad SCF arguments");
    for (auto& sp : subs)
      for (auto& q : sp->kp) REQ(q.have_orbitals, FDE_EINVAL, "orbitals of every subsystem must be set");
    ensure_vloc();
    const size_t ns = subs.size();
    frozen.ensure(ns * nr);  // the input densities rho_in of every subsystem
    for (size_t I = 0; I < ns; ++I)
      CK(cudaMemcpyAsync(frozen.p + I * nr, subs[I]->rho.p, nr * sizeof(double), cudaMemcpyDeviceToDevice, st));
    fresh.ensure(ns * nr);  // the output densities, stacked for the joint mixing
    pulay_reset(hist_all);
    // Every refresh step mixes the output densities of eigensolves that start from the previous
    // step's orbitals, so their residual floor becomes the density residual's floor (about 30
    // times the eigensolver tolerance on the two-layer slab's Methfessel-Paxton meshes): FP64
    // solves go to 1/100 of tol to let the density residual reach 10 tol.
    const double dtol = sizeof(T) == 8 ? std::max(1e-12, std::min(1e-6, 0.01 * tol)) : davidson_tol(tol);
    std::vector<double> dres_prev(ns, 1.0), dres(ns, 0.0);
    double Fprev = 0;
    bool have_prev = false;
    fde_energies en{};
    for (int it = 1; it <= max_scf; ++it) {
      for (size_t I = 0; I < ns; ++I)
        CK(cudaMemcpyAsync(subs[I]->rho.p, frozen.p + I * nr, nr * sizeof(double), cudaMemcpyDeviceToDevice, st));
      grid_pass(true, false, -1);
      for (size_t I = 0; I < ns; ++I) {
        Sub<T>& s = *subs[I];
        for (int k = 0; k < s.nk; ++k) {
          int its = 0;
          subspace_solve((int)I, k, std::max(dtol, std::min(1e-3, 1e-4 * dres_prev[I])), 60, &its, precond_mode);
          davidson_iters += its;
        }
        occupations(s);
        density_from_orbitals(s, s.rho.p);
      }
      sync();
      energy(&en);
      double worst = 0;
      for (size_t I = 0; I < ns; ++I) {
        dres[I] = integrate_absdiff(subs[I]->rho.p, frozen.p + I * nr);
        dres_prev[I] = dres[I];
        worst = std::max(worst, dres[I]);
      }
      en.iters = it;
      en.dE = have_prev ? en.F_fde - Fprev : 0.0;
      REQ(std::isfinite(en.F_fde), FDE_ENONFINITE, "non-finite energy");
      if (trace_level() > 0)
        fprintf(stderr, "[fde] refresh it %d F %.12f dE %.3e max drho %.3e eig_iters %lld\n", it, en.F_fde, en.dE,
                worst, davidson_iters);
      if (have_prev && fabs(en.dE) < tol && worst < dres_tol(tol)) {
        grid_pass(true, false, -1);  // potentials of the returned densities
        if (out) *out = en;
        return FDE_OK;
      }
      Fprev = en.F_fde;
      have_prev = true;
      for (size_t I = 0; I < ns; ++I)
        CK(cudaMemcpyAsync(fresh.p + I * nr, subs[I]->rho.p, nr * sizeof(double), cudaMemcpyDeviceToDevice, st));
      pulay(hist_all, frozen.p, fresh.p, (long long)ns * nr);
    }
    grid_pass(true, false, -1);
    if (out) *out = en;
    return FDE_ENOCONV;
  }

  // <Delta rho> = 1/2 int |rho - rho_ref| with rho = sum_I rho_I (Computational Details).
  double delta_rho(const double* d_ref) override {
    REQ(d_ref, FDE_EINVAL, "null reference density");
    REQ(!subs.empty(), FDE_EINVAL, "no subsystems");
    sum_densities();
    return 0.5 * integrate_absdiff(rho_tot.p, d_ref);
  }
};

template <> void EngineT<double>::convert_in(const double2* a, double2* b, size_t n) {
  launch_convert_c<double, double>(a, b, n, st);
}
template <> void EngineT<float>::convert_in(const double2* a, float2* b, size_t n) {
  launch_convert_c<double, float>(a, b, n, st);
}
template <> void EngineT<double>::convert_out(const double2* a, double2* b, size_t n) {
  launch_convert_c<double, double>(a, b, n, st);
}
template <> void EngineT<float>::convert_out(const float2* a, double2* b, size_t n) {
  launch_convert_c<float, double>(a, b, n, st);
}
}  // namespace fde

// ---- C ABI ------------------------------------------------------------------------------------
// A subsystem descriptor with its own copies of the caller's arrays.
struct SubsysCopy {
  fde_subsys_desc d{};
  std::vector<double> pos, Z, sigma, D, Qa, kpts, wk;
  explicit SubsysCopy(const fde_subsys_desc& s) : d(s) {
    pos.assign(s.pos, s.pos + 3 * s.natoms);
    Z.assign(s.Z, s.Z + s.natoms);
    if (s.nproj_per_atom > 0) {
      sigma.assign(s.proj_sigma, s.proj_sigma + s.nproj_per_atom);
      D.assign(s.proj_D, s.proj_D + s.nproj_per_atom * s.nproj_per_atom);
    }
    if (s.aug_sigma > 0 && s.proj_Q && s.nproj_per_atom > 0)
      Qa.assign(s.proj_Q, s.proj_Q + s.nproj_per_atom * s.nproj_per_atom);
    kpts.assign(s.kpts, s.kpts + 3 * s.nk);
    wk.assign(s.wk, s.wk + s.nk);
    d.proj_Q = Qa.empty() ? nullptr : Qa.data();
    d.pos = pos.data();
    d.Z = Z.data();
    d.proj_sigma = sigma.empty() ? nullptr : sigma.data();
    d.proj_D = D.empty() ? nullptr : D.data();
    d.kpts = kpts.data();
    d.wk = wk.data();
  }
};

struct fde_ctx {
  std::unique_ptr<fde::Engine> eng;    // working precision
  // FP64 refinement engine of a mixed context: built on first use (a mixed freeze-and-thaw
  // cycle or refreshed SCF) from the stored descriptors, so that mixed contexts whose FP64
  // plane would not fit in shared memory still run everything else
  std::unique_ptr<fde::Engine> eng64;
  fde_cell_desc cell{};
  fde_func_desc func{};
  std::vector<std::unique_ptr<SubsysCopy>> subs;
  std::vector<int> sym_ops;
  cudaStream_t stream = nullptr;
  std::string err;
  fde_prec prec;
  fde::Profiler prof;
};

namespace fde {

// The FP64 engine of a mixed context, created on first use.
static Engine& engine64(fde_ctx* c) {
  if (!c->eng64) {
    std::unique_ptr<Engine> e(new EngineT<double>(&c->cell, &c->func, c->stream));
    for (auto& sc : c->subs) e->add_subsystem(&sc->d);
    if (!c->sym_ops.empty()) e->set_symmetry((int)c->sym_ops.size(), c->sym_ops.data());
    c->eng64 = std::move(e);
  }
  return *c->eng64;
}

// Copy densities, orbitals, eigenvalues, occupations and entropies of every subsystem from
// one engine to another (the precisions may differ; orbitals pass through FP64).
static void transfer_state(Engine& from, Engine& to, cudaStream_t st) {
  const int ns = from.nsub();
  const long long nr = from.grid_points();
  DBuf<double> rho;
  rho.alloc(nr);
  for (int I = 0; I < ns; ++I) {
    from.get_density(I, rho.p);
    to.set_density(I, rho.p, 1);
    int nb, nk;
    from.shape(I, &nb, &nk);
    for (int k = 0; k < nk; ++k) {
      DBuf<double2> psi;
      psi.alloc((size_t)nb * from.npw(I, k));
      std::vector<double> eig(nb), occ(nb);
      from.get_orbitals(I, k, (double*)psi.p, eig.data(), occ.data());
      to.set_orbitals(I, k, (const double*)psi.p);
      to.set_eig_occ(I, k, eig.data(), occ.data());
      CK(cudaStreamSynchronize(st));
    }
    to.set_subsystem_entropy(I, from.subsystem_entropy(I));
  }
  CK(cudaStreamSynchronize(st));
}

// Mixed-precision freeze-and-thaw cycle: the FP32 engine runs the cycle to a relaxed
// tolerance, then the FP64 engine repeats the same cycle (same frozen densities) warm-
// started from the FP32 densities and orbitals to the requested tolerance, and the result
// is copied back to the FP32 engine.
static fde_status mixed_cycle(fde_ctx* c, double tol, int max_scf, fde_energies* out, cudaStream_t st) {
  Engine& lo = *c->eng;
  Engine& hi = engine64(c);
  const int ns = lo.nsub();
  const long long nr = lo.grid_points();
  DBuf<double> start;
  start.alloc((size_t)ns * nr);
  for (int I = 0; I < ns; ++I) {
    lo.get_density(I, start.p + I * nr);
    hi.set_density(I, start.p + I * nr, 1);
  }
  fde_energies e1{};
  const fde_status s1 = lo.freeze_thaw(std::max(tol, 1e-5), max_scf, &e1, nullptr);
  if (s1 != FDE_OK && s1 != FDE_ENOCONV) return s1;
  // orbitals of the FP32 result into the FP64 engine; its densities stay the frozen ones
  for (int I = 0; I < ns; ++I) {
    lo.get_density(I, start.p + I * nr);
    int nb, nk;
    lo.shape(I, &nb, &nk);
    for (int k = 0; k < nk; ++k) {
      DBuf<double2> psi;
      psi.alloc((size_t)nb * lo.npw(I, k));
      std::vector<double> eig(nb), occ(nb);
      lo.get_orbitals(I, k, (double*)psi.p, eig.data(), occ.data());
      hi.set_orbitals(I, k, (const double*)psi.p);
      hi.set_eig_occ(I, k, eig.data(), occ.data());
      CK(cudaStreamSynchronize(st));
    }
    hi.set_subsystem_entropy(I, lo.subsystem_entropy(I));
  }
  CK(cudaStreamSynchronize(st));
  fde_energies e2{};
  const fde_status s2 = hi.freeze_thaw(tol, max_scf, &e2, start.p);
  transfer_state(hi, lo, st);
  lo.build_vemb(nullptr, nullptr);
  lo.sync();
  if (out) {
    *out = e2;
    out->iters = e1.iters + e2.iters;
  }
  return s2;
}

// Mixed-precision refreshed SCF: the FP32 engine converges to a relaxed tolerance, the FP64
// engine continues from its densities and orbitals to the requested one, and the result is
// copied back to the FP32 engine.
static fde_status mixed_refresh(fde_ctx* c, double tol, int max_scf, fde_energies* out, cudaStream_t st) {
  Engine& lo = *c->eng;
  Engine& hi = engine64(c);
  fde_energies e1{};
  const fde_status s1 = lo.scf_refresh(std::max(tol, 1e-5), max_scf, &e1);
  if (s1 != FDE_OK && s1 != FDE_ENOCONV) return s1;
  transfer_state(lo, hi, st);
  fde_energies e2{};
  const fde_status s2 = hi.scf_refresh(tol, max_scf, &e2);
  transfer_state(hi, lo, st);
  lo.build_vemb(nullptr, nullptr);
  lo.sync();
  if (out) {
    *out = e2;
    out->iters = e1.iters + e2.iters;
  }
  return s2;
}

}  // namespace fde

template <typename F> static fde_status guard(fde_ctx* c, F&& f) {
  if (!c) return FDE_EINVAL;
  fde::tl_prof = &c->prof;
  fde_status r;
  try {
    c->err.clear();
    r = f();
  } catch (fde::Err& e) {
    c->err = e.msg;
    r = e.st;
  } catch (std::exception& e) {
    c->err = e.what();
    r = FDE_ENOMEM;
  }
  fde::tl_prof = nullptr;
  return r;
}

extern "C" {

fde_status fde_create(const fde_cell_desc* cell, const fde_func_desc* func, fde_prec prec, void* cuda_stream,
                      fde_ctx** out) {
  if (!cell || !func || !out) return FDE_EINVAL;
  *out = nullptr;
  if (prec != FDE_PREC_FP64 && prec != FDE_PREC_MIXED) return FDE_EINVAL;
  fde_ctx* c = new fde_ctx();
  c->prec = prec;
  fde_status s = guard(c, [&]() {
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (prec == FDE_PREC_FP64) c->eng.reset(new fde::EngineT<double>(cell, func, st));
    else {
      c->eng.reset(new fde::EngineT<float>(cell, func, st));
      c->cell = *cell;
      c->func = *func;
    }
    c->stream = st;
    return FDE_OK;
  });
  if (s != FDE_OK) {
    fprintf(stderr, "fde_create: %s\n", c->err.c_str());
    delete c;
    return s;
  }
  *out = c;
  return FDE_OK;
}

fde_status fde_add_subsystem(fde_ctx* c, const fde_subsys_desc* d, int* id) {
  return guard(c, [&]() {
    const int i = c->eng->add_subsystem(d);
    if (c->prec == FDE_PREC_MIXED) {
      c->subs.emplace_back(new SubsysCopy(*d));
      if (c->eng64) c->eng64->add_subsystem(d);
    }
    if (id) *id = i;
    return FDE_OK;
  });
}
fde_status fde_get_basis(fde_ctx* c, int sub, int k, int* npw, int* miller) {
  return guard(c, [&]() { c->eng->get_basis(sub, k, npw, miller); return FDE_OK; });
}
fde_status fde_set_density(fde_ctx* c, int sub, const double* rho, int on_device) {
  return guard(c, [&]() { c->eng->set_density(sub, rho, on_device); return FDE_OK; });
}
fde_status fde_get_density(fde_ctx* c, int sub, double* d_rho) {
  return guard(c, [&]() { c->eng->get_density(sub, d_rho); return FDE_OK; });
}
fde_status fde_build_vemb(fde_ctx* c, double* d_out, fde_energies* e) {
  return guard(c, [&]() { c->eng->build_vemb(d_out, e); return FDE_OK; });
}
fde_status fde_set_veff(fde_ctx* c, int sub, const double* d_v) {
  return guard(c, [&]() { c->eng->set_veff(sub, d_v); return FDE_OK; });
}
fde_status fde_apply_h(fde_ctx* c, int sub, int k, const void* psi, void* hpsi, int nb) {
  return guard(c, [&]() { c->eng->apply_h(sub, k, psi, hpsi, nb); return FDE_OK; });
}
fde_status fde_apply_s(fde_ctx* c, int sub, int k, const void* psi, void* spsi, int nb) {
  return guard(c, [&]() { c->eng->apply_s_dev(sub, k, psi, spsi, nb); return FDE_OK; });
}
fde_status fde_apply_h_host(fde_ctx* c, int sub, int k, const double* psi, double* hpsi, int nb) {
  return guard(c, [&]() { c->eng->apply_h_host(sub, k, psi, hpsi, nb); return FDE_OK; });
}
fde_status fde_apply_h_all(fde_ctx* c) {
  return guard(c, [&]() { c->eng->apply_h_all(); return FDE_OK; });
}
fde_status fde_init_orbitals(fde_ctx* c, int sub, int k, const double* raw) {
  return guard(c, [&]() { c->eng->init_orbitals(sub, k, raw); return FDE_OK; });
}
fde_status fde_set_orbitals(fde_ctx* c, int sub, int k, const double* d_psi) {
  return guard(c, [&]() { c->eng->set_orbitals(sub, k, d_psi); return FDE_OK; });
}
fde_status fde_get_orbitals(fde_ctx* c, int sub, int k, double* d_psi, double* eig, double* occ) {
  return guard(c, [&]() { c->eng->get_orbitals(sub, k, d_psi, eig, occ); return FDE_OK; });
}
fde_status fde_subspace_solve(fde_ctx* c, int sub, int k, double tol, int max_iter, int precond, int* iters) {
  return guard(c, [&]() {
    if (precond != FDE_PRECOND_TPA && precond != FDE_PRECOND_LEARNED)
      throw fde::Err{FDE_EUNSUPPORTED, "unknown preconditioner"};
    return c->eng->subspace_solve(sub, k, tol, max_iter, iters, precond);
  });
}
fde_status fde_update_density(fde_ctx* c, int sub) {
  return guard(c, [&]() { c->eng->update_density(sub); return FDE_OK; });
}
fde_status fde_energy(fde_ctx* c, fde_energies* out) {
  return guard(c, [&]() { c->eng->energy(out); return FDE_OK; });
}
fde_status fde_scf_subsystem(fde_ctx* c, int sub, double tol, int max_scf, fde_energies* out) {
  return guard(c, [&]() { return c->eng->scf_subsystem(sub, tol, max_scf, out); });
}
fde_status fde_freeze_thaw_cycle(fde_ctx* c, double tol, int max_scf, fde_energies* out) {
  return guard(c, [&]() {
    if (c->prec == FDE_PREC_MIXED) return fde::mixed_cycle(c, tol, max_scf, out, c->stream);
    return c->eng->freeze_thaw(tol, max_scf, out, nullptr);
  });
}
fde_status fde_scf_refresh(fde_ctx* c, double tol, int max_scf, fde_energies* out) {
  return guard(c, [&]() {
    if (c->prec == FDE_PREC_MIXED) return fde::mixed_refresh(c, tol, max_scf, out, c->stream);
    return c->eng->scf_refresh(tol, max_scf, out);
  });
}
fde_status fde_set_symmetry(fde_ctx* c, int nops, const int* ops) {
  return guard(c, [&]() {
    c->eng->set_symmetry(nops, ops);
    if (c->prec == FDE_PREC_MIXED) c->sym_ops.assign(ops, ops + nops);
    if (c->eng64) c->eng64->set_symmetry(nops, ops);
    return FDE_OK;
  });
}
fde_status fde_delta_rho(fde_ctx* c, const double* d_rho_ref, double* out) {
  return guard(c, [&]() {
    if (!out) throw fde::Err{FDE_EINVAL, "null output"};
    *out = c->eng->delta_rho(d_rho_ref);
    return FDE_OK;
  });
}
fde_status fde_set_precond(fde_ctx* c, int precond) {
  return guard(c, [&]() { c->eng->set_precond_mode(precond); return FDE_OK; });
}
fde_status fde_precond_set_weights(fde_ctx* c, const float* h) {
  return guard(c, [&]() { c->eng->precond_set_weights(h); return FDE_OK; });
}
fde_status fde_precond_get_weights(fde_ctx* c, float* h, float* hb) {
  return guard(c, [&]() { c->eng->precond_get_weights(h, hb); return FDE_OK; });
}
fde_status fde_precond_harvest(fde_ctx* c, int sub, int k, const double* raw, int n) {
  return guard(c, [&]() { c->eng->precond_harvest(sub, k, raw, n); return FDE_OK; });
}
fde_status fde_precond_add_pairs(fde_ctx* c, int sub, int k, int n, const double* r, const double* d,
                                 const double* tband) {
  return guard(c, [&]() { c->eng->precond_add_pairs(sub, k, n, r, d, tband); return FDE_OK; });
}
fde_status fde_get_hpsi(fde_ctx* c, int sub, int k, double* d_hpsi) {
  return guard(c, [&]() { c->eng->get_hpsi(sub, k, d_hpsi); return FDE_OK; });
}
fde_status fde_hot_step_host(fde_ctx* c, const double* const* h_rho, const double* const* h_psi,
                             double* const* h_hpsi) {
  return guard(c, [&]() {
    c->eng->hot_step_host(h_rho, h_psi, h_hpsi);
    return FDE_OK;
  });
}
fde_status fde_hot_step(fde_ctx* c, int use_graph) {
  return guard(c, [&]() {
    if (use_graph && c->stream == nullptr)
      throw fde::Err{FDE_EINVAL, "graph replay needs a non-default context stream"};
    c->eng->hot_step(use_graph != 0);
    return FDE_OK;
  });
}
fde_status fde_precond_record(fde_ctx* c, int iterations) {
  return guard(c, [&]() { c->eng->set_precond_record(iterations); return FDE_OK; });
}
fde_status fde_precond_clear(fde_ctx* c) {
  return guard(c, [&]() { c->eng->precond_clear(); return FDE_OK; });
}
fde_status fde_precond_loss_grad(fde_ctx* c, double* grad, double* loss) {
  return guard(c, [&]() { c->eng->precond_loss_grad(grad, loss); return FDE_OK; });
}
fde_status fde_precond_train(fde_ctx* c, int steps, double lr, double* loss_first, double* loss_last) {
  return guard(c, [&]() { c->eng->precond_train(steps, lr, loss_first, loss_last); return FDE_OK; });
}
fde_status fde_precond_apply(fde_ctx* c, int sub, int k, const void* d_r, void* d_w, int nb, const double* tband) {
  return guard(c, [&]() { c->eng->precond_apply(sub, k, d_r, d_w, nb, tband); return FDE_OK; });
}
fde_status fde_get_stats(fde_ctx* c, long long* davidson_iters, long long* hpsi_bands) {
  return guard(c, [&]() { c->eng->stats(davidson_iters, hpsi_bands); return FDE_OK; });
}
fde_status fde_gemm_hn_f32(fde_ctx* c, const void* d_A, int lda, const void* d_B, int ldb, int m, int n, int K,
                           double* d_C, int ldc, int path) {
  return guard(c, [&]() {
    using fde::Err;
    if (!d_A || !d_B || !d_C || m <= 0 || n <= 0 || K <= 0 || lda < K || ldb < K || ldc < n ||
        (path != 0 && path != 1 && path != 3))
      throw fde::Err{FDE_EINVAL, "bad product arguments"};
    fde::DBuf<double2> work;
    work.alloc(fde::gemm_hn_work(m, n, K));
    const int saved = fde::gemm_hn_path();
    fde::set_gemm_hn_path(path);
    fde::launch_gemm_hn<float>((const float2*)d_A, lda, (const float2*)d_B, ldb, m, n, K, (double2*)d_C, ldc,
                               work.p, c->stream);
    fde::set_gemm_hn_path(saved);
    CK(cudaStreamSynchronize(c->stream));
    if (fde::gemm_tc_take_status(c->stream) & fde::ST_TIMEOUT)
      throw fde::Err{FDE_ETIMEOUT, "a tensor-core product timed out waiting for its MMAs"};
    return FDE_OK;
  });
}

fde_status fde_gemm_rot_f32(fde_ctx* c, const void* d_X, int ldx, const double* d_U, int ldu, int m, int n, int K,
                            void* d_Y, int ldy, double alpha, double beta, int path) {
  return guard(c, [&]() {
    using fde::Err;
    if (!d_X || !d_U || !d_Y || m <= 0 || n <= 0 || K <= 0 || ldx < K || ldy < K || ldu < n ||
        (path != 0 && path != 1 && path != 3))
      throw fde::Err{FDE_EINVAL, "bad combination arguments"};
    const int saved = fde::gemm_hn_path();
    fde::set_gemm_hn_path(path);
    fde::launch_gemm_rot<float>((const float2*)d_X, ldx, (const double2*)d_U, ldu, m, n, K, (float2*)d_Y, ldy,
                                alpha, beta, c->stream, path != 0);
    fde::set_gemm_hn_path(saved);
    CK(cudaStreamSynchronize(c->stream));
    if (fde::gemm_tc_take_status(c->stream) & fde::ST_TIMEOUT)
      throw fde::Err{FDE_ETIMEOUT, "a tensor-core combination timed out waiting for its MMAs"};
    return FDE_OK;
  });
}

int fde_tuned_plane_variant(int n1, int n3) { return fde::query_plane_variant(n1, n3); }
fde_status fde_pin_plane_variant(int variant) { return fde::pin_plane_variant(variant) ? FDE_OK : FDE_EINVAL; }

fde_status fde_set_tc_wait_limit(long long polls) {
  return fde::set_tc_stage_spin(polls) && fde::set_precond_tc_spin(polls) ? FDE_OK : FDE_ECUDA;
}

fde_status fde_set_precond_path(int path) {
  if (path != 0 && path != 1) return FDE_EINVAL;
  fde::set_precond_tensor_cores(path == 1);
  return FDE_OK;
}

fde_status fde_set_gemm_path(int path) {
  if (path != 0 && path != 1 && path != 3) return FDE_EINVAL;
  fde::set_gemm_hn_path(path);
  return FDE_OK;
}

fde_status fde_dense_eigh(fde_ctx* c, int n, const double* d_A, int nvec, double* d_w, double* d_V) {
  return guard(c, [&]() {
    using fde::Err;
    if (n <= 0 || n > 1024 || nvec < 0 || nvec > n || !d_A || !d_w || !d_V)
      throw fde::Err{FDE_EINVAL, "bad eigensolver arguments"};
    fde::DBuf<double2> a;
    fde::DBuf<double> wk;
    a.alloc((size_t)n * n);
    wk.alloc(fde::heev_work_doubles(n, nvec));
    CK(cudaMemcpyAsync(a.p, d_A, (size_t)n * n * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
    fde::launch_heev(a.p, n, nvec, d_w, (double2*)d_V, wk.p, c->stream);
    CK(cudaStreamSynchronize(c->stream));
    return FDE_OK;
  });
}
fde_status fde_fft3d(fde_ctx* c, void* d_data, int sign) {
  return guard(c, [&]() { c->eng->fft3d(d_data, sign); return FDE_OK; });
}
fde_status fde_fft3d_f64(fde_ctx* c, double* d_data, int sign, int arith) {
  return guard(c, [&]() { c->eng->fft3d_f64((double2*)d_data, sign, arith); return FDE_OK; });
}
fde_status fde_sync(fde_ctx* c) {
  return guard(c, [&]() { c->eng->sync(); return FDE_OK; });
}
fde_status fde_profile_enable(fde_ctx* c, int enable) {
  return guard(c, [&]() {
    if (enable < 0 || enable > 2) throw fde::Err{FDE_EINVAL, "profiling level must be 0, 1 or 2"};
    c->eng->sync();
    c->prof.reset();
    c->prof.on = enable != 0;
    c->prof.level = enable == 2 ? 2 : 1;
    return FDE_OK;
  });
}
fde_status fde_profile_get(fde_ctx* c, const char* kernel, int* launches, double* total_ms) {
  return guard(c, [&]() {
    if (!kernel || !launches || !total_ms) throw fde::Err{FDE_EINVAL, "null argument"};
    c->prof.get(kernel, launches, total_ms);
    return FDE_OK;
  });
}
fde_status fde_launch_count(fde_ctx* c, long long* launches) {
  return guard(c, [&]() {
    if (!launches) throw fde::Err{FDE_EINVAL, "null argument"};
    *launches = c->prof.launches;
    return FDE_OK;
  });
}
const char* fde_last_error(const fde_ctx* c) { return c ? c->err.c_str() : "null context"; }
fde_status fde_destroy(fde_ctx* c) {
  if (!c) return FDE_EINVAL;
  delete c;
  return FDE_OK;
}

}  // extern "C"
