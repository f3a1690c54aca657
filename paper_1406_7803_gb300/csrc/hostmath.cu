// hostmath.cu -- host-side numerics of the engine (hostmath.h) and their C-ABI entry points.
//   * plane-wave sphere |k + G|^2 / 2 <= E_cut (Sec. 2: plane-wave expansion of the subsystem
//     orbitals; the full sphere, evaluated in FP64 from integer Miller indices);
//   * Ewald sum with a neutralising background for the nuclear repulsion V_NN of Eq. E_FDE;
//   * occupations with 2 sum_k w_k sum_j n_jk = N_I (Sec. 2), Methfessel-Paxton (the paper's),
//     Gaussian or Fermi-Dirac smearing for metallic subsystems (Computational Details) and the
//     entropy term of each;
//   * Pulay (DIIS) mixing coefficients of the subsystem SCF (the paper is silent on mixing);
//   * Monkhorst-Pack meshes reduced by time reversal and the cell's mirror symmetries
//     (Computational Details: 2 x 2 x 1 Monkhorst-Pack sampling of the periodic systems).
#include <math.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "fde.h"
#include "hostmath.h"

namespace fde {

void sphere_miller(const double L[3], const double kfrac[3], double ecut, std::vector<int>& miller,
                   std::vector<double>& kin, double kc[3]) {
  double B[3];
  for (int j = 0; j < 3; ++j) B[j] = 2.0 * M_PI * (1.0 / L[j]);
  for (int c = 0; c < 3; ++c) kc[c] = kfrac[c] * B[c];
  const double knorm = sqrt(kc[0] * kc[0] + kc[1] * kc[1] + kc[2] * kc[2]);
  const double qmax = sqrt(2.0 * ecut) + knorm;
  int lim[3];
  for (int j = 0; j < 3; ++j) lim[j] = (int)ceil(qmax * L[j] / (2.0 * M_PI)) + 1;
  miller.clear();
  kin.clear();
  for (int m1 = -lim[0]; m1 <= lim[0]; ++m1)
    for (int m2 = -lim[1]; m2 <= lim[1]; ++m2)
      for (int m3 = -lim[2]; m3 <= lim[2]; ++m3) {
        const double q0 = kc[0] + (double)m1 * B[0], q1 = kc[1] + (double)m2 * B[1], q2 = kc[2] + (double)m3 * B[2];
        const double kk = 0.5 * (q0 * q0 + q1 * q1 + q2 * q2);
        if (kk <= ecut) {
          miller.push_back(m1);
          miller.push_back(m2);
          miller.push_back(m3);
          kin.push_back(kk);
        }
      }
}

double ewald_energy(const double Lc[3], const std::vector<double>& pos, const std::vector<double>& Z) {
  double A[3][3] = {{Lc[0], 0, 0}, {0, Lc[1], 0}, {0, 0, Lc[2]}};
  double B[3][3] = {{2 * M_PI / Lc[0], 0, 0}, {0, 2 * M_PI / Lc[1], 0}, {0, 0, 2 * M_PI / Lc[2]}};
  const double omega = Lc[0] * Lc[1] * Lc[2];
  const int n = (int)Z.size();
  const double eta = sqrt(M_PI) / cbrt(omega);
  const double x = sqrt(-log(1e-16));
  const double rmax = x / eta + 1.0, gmax = 2.0 * eta * x + 1.0;
  int nl[3], ng[3];
  for (int j = 0; j < 3; ++j) {
    const double bn = sqrt(B[j][0] * B[j][0] + B[j][1] * B[j][1] + B[j][2] * B[j][2]);
    const double an = sqrt(A[j][0] * A[j][0] + A[j][1] * A[j][1] + A[j][2] * A[j][2]);
    nl[j] = (int)ceil(rmax * bn / (2 * M_PI)) + 1;
    ng[j] = (int)ceil(gmax * an / (2 * M_PI)) + 1;
  }
  double er = 0.0;
  for (int a = -nl[0]; a <= nl[0]; ++a)
    for (int b = -nl[1]; b <= nl[1]; ++b)
      for (int c = -nl[2]; c <= nl[2]; ++c) {
        double Lv[3];
        for (int d = 0; d < 3; ++d) Lv[d] = a * A[0][d] + b * A[1][d] + c * A[2][d];
        for (int i = 0; i < n; ++i)
          for (int j = 0; j < n; ++j) {
            if (a == 0 && b == 0 && c == 0 && i == j) continue;
            double r2 = 0;
            for (int d = 0; d < 3; ++d) {
              const double dd = pos[3 * i + d] - pos[3 * j + d] + Lv[d];
              r2 += dd * dd;
            }
            const double r = sqrt(r2);
            if (r < rmax) er += 0.5 * Z[i] * Z[j] * erfc(eta * r) / r;
          }
      }
  double eg = 0.0;
  for (int a = -ng[0]; a <= ng[0]; ++a)
    for (int b = -ng[1]; b <= ng[1]; ++b)
      for (int c = -ng[2]; c <= ng[2]; ++c) {
        double G[3];
        for (int d = 0; d < 3; ++d) G[d] = a * B[0][d] + b * B[1][d] + c * B[2][d];
        const double g2 = G[0] * G[0] + G[1] * G[1] + G[2] * G[2];
        if (g2 <= 0 || g2 >= gmax * gmax) continue;
        double sr = 0, si = 0;
        for (int i = 0; i < n; ++i) {
          const double ph = G[0] * pos[3 * i] + G[1] * pos[3 * i + 1] + G[2] * pos[3 * i + 2];
          sr += Z[i] * cos(ph);
          si += Z[i] * sin(ph);
        }
        eg += exp(-g2 / (4 * eta * eta)) / g2 * (sr * sr + si * si);
      }
  eg *= 2.0 * M_PI / omega;
  double z2 = 0, zs = 0;
  for (int i = 0; i < n; ++i) {
    z2 += Z[i] * Z[i];
    zs += Z[i];
  }
  return er + eg - eta / sqrt(M_PI) * z2 - M_PI * zs * zs / (2.0 * omega * eta * eta);
}

static inline double fermi(double x) {  // 1 / (1 + e^x)
  if (x > 0) {
    const double e = exp(-x);
    return e / (1.0 + e);
  }
  return 1.0 / (1.0 + exp(x));
}

// Occupation f(x) and entropy-like term s(x) of one state at x = (e - mu) / sigma.  s is the
// function for which the free energy E - sigma 2 sum_k w_k sum_j s(x_jk) is variational in
// the occupations: s'(x) = x f'(x), s(-inf) = 0.
//   Fermi-Dirac: f = 1 / (1 + e^x), s = -[f ln f + (1 - f) ln(1 - f)];
//   Gaussian (Methfessel-Paxton order 0): f = erfc(x) / 2, s = e^{-x^2} / (2 sqrt(pi));
//   Methfessel-Paxton order 1 (Computational Details: the metallic subsystems' smearing):
//     the Gaussian delta corrected by its first Hermite term, A_1 H_2(x) e^{-x^2} with
//     A_1 = -1 / (4 sqrt(pi)), integrates to f = erfc(x) / 2 - x e^{-x^2} / (2 sqrt(pi)) and
//     s = A_1 H_2(x) e^{-x^2} / 2 = (1 - 2 x^2) e^{-x^2} / (4 sqrt(pi)).
static inline void smear(int kind, double x, double* f, double* s) {
  const double isp = 0.5641895835477562869;  // 1 / sqrt(pi)
  if (kind == FDE_SMEAR_FERMI) {
    const double n = fermi(x);
    double t = 0;
    if (n > 0) t += n * log(n);
    if (n < 1) t += (1 - n) * log(1 - n);
    *f = n;
    *s = -t;
    return;
  }
  const double g = exp(-x * x);
  if (kind == FDE_SMEAR_GAUSS) {
    *f = 0.5 * erfc(x);
    *s = 0.5 * isp * g;
    return;
  }
  *f = 0.5 * erfc(x) - 0.5 * isp * x * g;
  *s = 0.25 * isp * (1.0 - 2.0 * x * x) * g;
}

bool occupations_host(int nk, int nb, const double* eig, const double* wk, double nelec, double sigma, double* occ,
                      double* mu, double* ts, int kind) {
  if (kind != FDE_SMEAR_FERMI && kind != FDE_SMEAR_MP && kind != FDE_SMEAR_GAUSS) return false;
  if (nk <= 0 || nb <= 0 || !eig || !wk || !occ) return false;
  if (sigma <= 0) {
    const int no = (int)llround(nelec / 2.0);
    if (nk != 1 || no < 0 || no > nb || fabs(nelec / 2.0 - no) > 1e-12) return false;
    std::vector<int> order(nb);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return eig[a] < eig[b]; });
    for (int j = 0; j < nb; ++j) occ[j] = 0.0;
    for (int j = 0; j < no; ++j) occ[order[j]] = 1.0;
    if (mu) *mu = no ? eig[order[no - 1]] : eig[order[0]];
    if (ts) *ts = 0.0;
    return true;
  }
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < nk * nb; ++i) {
    lo = std::min(lo, eig[i]);
    hi = std::max(hi, eig[i]);
  }
  lo -= 40.0 * sigma;
  hi += 40.0 * sigma;
  double m = 0.5 * (lo + hi);
  for (int it = 0; it < 300; ++it) {
    m = 0.5 * (lo + hi);
    double n = 0, f, sj;
    for (int k = 0; k < nk; ++k)
      for (int j = 0; j < nb; ++j) {
        smear(kind, (eig[k * nb + j] - m) / sigma, &f, &sj);
        n += 2.0 * wk[k] * f;
      }
    if (fabs(n - nelec) < 1e-13) break;
    if (n < nelec) lo = m; else hi = m;
  }
  double S = 0;
  for (int k = 0; k < nk; ++k)
    for (int j = 0; j < nb; ++j) {
      double f, sj;
      smear(kind, (eig[k * nb + j] - m) / sigma, &f, &sj);
      occ[k * nb + j] = f;
      S += 2.0 * wk[k] * sj;
    }
  if (mu) *mu = m;
  if (ts) *ts = sigma * S;
  return true;
}

// ---- Brillouin-zone sampling --------------------------------------------------------------------
// Monkhorst-Pack mesh: k_j = (2 r_j - q_j - 1 + shift_j) / (2 q_j), r_j = 1..q_j, crystal coordinates,
// enumerated with the first axis slowest.  Two points are the same when they differ by a
// reciprocal lattice vector (integer crystal coordinates).
static bool same_k(const double* a, const double* b) {
  for (int c = 0; c < 3; ++c) {
    const double d = a[c] - b[c];
    if (fabs(d - nearbyint(d)) > 1e-9) return false;
  }
  return true;
}

bool kmesh_host(const int q[3], const double shift[3], int time_reversal, int nops, const int* ops,
                std::vector<double>& kpts, std::vector<double>& wk) {
  for (int c = 0; c < 3; ++c)
    if (q[c] <= 0 || q[c] > 64) return false;
  if (nops < 0 || (nops > 0 && !ops)) return false;
  std::vector<double> full;
  for (int a = 1; a <= q[0]; ++a)
    for (int b = 1; b <= q[1]; ++b)
      for (int c = 1; c <= q[2]; ++c) {
        const int r[3] = {a, b, c};
        for (int d = 0; d < 3; ++d) full.push_back((2.0 * r[d] - q[d] - 1.0 + (shift ? shift[d] : 0.0)) / (2.0 * q[d]));
      }
  const int n = (int)full.size() / 3;
  // images of a point: R k for every operation (identity included), and -R k with time reversal
  std::vector<int> opl(1, 0);
  for (int o = 0; o < nops; ++o) {
    if (ops[o] < 0 || ops[o] > 7) return false;
    if (std::find(opl.begin(), opl.end(), ops[o]) == opl.end()) opl.push_back(ops[o]);
  }
  std::vector<int> owner(n, -1);
  kpts.clear();
  wk.clear();
  for (int i = 0; i < n; ++i) {
    if (owner[i] >= 0) continue;
    const int id = (int)wk.size();
    int count = 0;
    for (int j = i; j < n; ++j) {
      if (owner[j] >= 0) continue;
      bool hit = false;
      for (int o : opl)
        for (int t = 0; t < (time_reversal ? 2 : 1) && !hit; ++t) {
          double img[3];
          for (int d = 0; d < 3; ++d) img[d] = ((o >> d) & 1 ? -1.0 : 1.0) * (t ? -1.0 : 1.0) * full[3 * i + d];
          hit = same_k(img, &full[3 * j]);
        }
      if (hit) {
        owner[j] = id;
        ++count;
      }
    }
    for (int d = 0; d < 3; ++d) kpts.push_back(full[3 * i + d]);
    wk.push_back((double)count / (double)n);
  }
  return true;
}

// Operations r -> R r about the origin, R = diag(+-1, +-1, +-1) (3-bit mask: bit c flips
// coordinate c), that map the atom set onto itself: every atom lands within tol (bohr, modulo
// the cell) on an atom of the same charge.  The identity (mask 0) is always first.
void symmetry_ops_host(const double L[3], int natoms, const double* pos, const double* Z, double tol,
                       std::vector<int>& ops) {
  ops.assign(1, 0);
  for (int m = 1; m < 8; ++m) {
    bool ok = true;
    for (int a = 0; a < natoms && ok; ++a) {
      double p[3];
      for (int d = 0; d < 3; ++d) p[d] = ((m >> d) & 1) ? -pos[3 * a + d] : pos[3 * a + d];
      bool found = false;
      for (int b = 0; b < natoms && !found; ++b) {
        if (Z[a] != Z[b]) continue;
        double r2 = 0;
        for (int d = 0; d < 3; ++d) {
          double x = p[d] - pos[3 * b + d];
          x -= L[d] * nearbyint(x / L[d]);
          r2 += x * x;
        }
        found = r2 <= tol * tol;
      }
      ok = found;
    }
    if (ok) ops.push_back(m);
  }
}

bool solve_dense(std::vector<double>& Am, std::vector<double>& b, int n) {
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(Am[r * n + c]) > fabs(Am[p * n + c])) p = r;
    if (fabs(Am[p * n + c]) < 1e-300) return false;
    if (p != c) {
      for (int k = 0; k < n; ++k) std::swap(Am[c * n + k], Am[p * n + k]);
      std::swap(b[c], b[p]);
    }
    for (int r = c + 1; r < n; ++r) {
      const double f = Am[r * n + c] / Am[c * n + c];
      for (int k = c; k < n; ++k) Am[r * n + k] -= f * Am[c * n + k];
      b[r] -= f * b[c];
    }
  }
  for (int c = n - 1; c >= 0; --c) {
    double v = b[c];
    for (int k = c + 1; k < n; ++k) v -= Am[c * n + k] * b[k];
    b[c] = v / Am[c * n + c];
  }
  return true;
}

bool pulay_coefficients(const double* ov, int m, double* coef) {
  // [ ov  1 ] [c]   [0]
  // [ 1^T 0 ] [l] = [1]
  std::vector<double> Am((size_t)(m + 1) * (m + 1), 0.0), b(m + 1, 0.0);
  for (int a = 0; a < m; ++a)
    for (int c = 0; c < m; ++c) Am[a * (m + 1) + c] = ov[a * m + c];
  for (int a = 0; a < m; ++a) Am[a * (m + 1) + m] = Am[m * (m + 1) + a] = 1.0;
  b[m] = 1.0;
  if (!solve_dense(Am, b, m + 1)) {
    for (int a = 0; a < m; ++a) coef[a] = 0.0;
    coef[m - 1] = 1.0;
    return false;
  }
  for (int a = 0; a < m; ++a) coef[a] = b[a];
  return true;
}

}  // namespace fde

// ---- C ABI (host only) --------------------------------------------------------------------------
fde_status fde_host_sphere(const double* lengths, const double* kfrac, double ecut, int* npw, int* miller,
                           double* kin) {
  if (!lengths || !kfrac || !npw || !(ecut > 0)) return FDE_EINVAL;
  for (int j = 0; j < 3; ++j)
    if (!(lengths[j] > 0)) return FDE_EINVAL;
  std::vector<int> m;
  std::vector<double> k;
  double kc[3];
  const int cap = *npw;
  fde::sphere_miller(lengths, kfrac, ecut, m, k, kc);
  *npw = (int)k.size();
  if ((miller || kin) && cap < *npw) return FDE_EINVAL;  // output buffers hold cap entries
  if (miller) std::copy(m.begin(), m.end(), miller);
  if (kin) std::copy(k.begin(), k.end(), kin);
  return FDE_OK;
}

fde_status fde_host_ewald(const double* lengths, int natoms, const double* pos, const double* Z, double* energy) {
  if (!lengths || natoms <= 0 || !pos || !Z || !energy) return FDE_EINVAL;
  for (int j = 0; j < 3; ++j)
    if (!(lengths[j] > 0)) return FDE_EINVAL;
  *energy = fde::ewald_energy(lengths, std::vector<double>(pos, pos + 3 * natoms), std::vector<double>(Z, Z + natoms));
  return FDE_OK;
}

fde_status fde_host_occupations(int nk, int nb, const double* eig, const double* wk, double nelec, double sigma,
                                int smearing_kind, double* occ, double* mu, double* ts) {
  return fde::occupations_host(nk, nb, eig, wk, nelec, sigma, occ, mu, ts, smearing_kind) ? FDE_OK : FDE_EINVAL;
}

fde_status fde_host_kmesh(const int* q, const double* shift, int time_reversal, int nops, const int* ops, int* nk,
                          double* kpts, double* wk) {
  if (!q || !nk) return FDE_EINVAL;
  std::vector<double> k, w;
  if (!fde::kmesh_host(q, shift, time_reversal, nops, ops, k, w)) return FDE_EINVAL;
  const int cap = *nk;
  *nk = (int)w.size();
  if ((kpts || wk) && cap < *nk) return FDE_EINVAL;
  if (kpts) std::copy(k.begin(), k.end(), kpts);
  if (wk) std::copy(w.begin(), w.end(), wk);
  return FDE_OK;
}

fde_status fde_host_symmetry_ops(const double* lengths, int natoms, const double* pos, const double* Z, double tol,
                                 int* nops, int* ops) {
  if (!lengths || natoms < 0 || (natoms > 0 && (!pos || !Z)) || !nops || !ops || !(tol >= 0)) return FDE_EINVAL;
  for (int j = 0; j < 3; ++j)
    if (!(lengths[j] > 0)) return FDE_EINVAL;
  std::vector<int> o;
  fde::symmetry_ops_host(lengths, natoms, pos, Z, tol, o);
  *nops = (int)o.size();
  std::copy(o.begin(), o.end(), ops);
  return FDE_OK;
}

fde_status fde_host_pulay(int m, const double* overlap, double* coef) {
  if (m <= 0 || !overlap || !coef) return FDE_EINVAL;
  return fde::pulay_coefficients(overlap, m, coef) ? FDE_OK : FDE_ENOCONV;
}
