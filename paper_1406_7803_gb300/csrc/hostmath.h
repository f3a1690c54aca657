// hostmath.h -- host-side numerics of the engine (no CUDA calls): the plane-wave sphere, the
// Ewald nuclear repulsion, occupations with the chemical potential, and the Pulay mixing
// coefficients.  The engine calls these functions; the C ABI exposes them (fde_host_*) so
// they can be checked on a machine without a GPU.
#pragma once

#include <vector>

namespace fde {

// Plane-wave sphere of an orthorhombic cell (edge lengths L[3], bohr) at the k-point kfrac
// (crystal coordinates): every Miller triple m with |k + G_m|^2 / 2 <= ecut, evaluated in
// FP64 from the integer indices, enumerated with m1 slowest and m3 fastest (ascending), so
// each (m1, m2) column is one contiguous run of m3.  miller gets 3 ints per plane wave, kin
// the kinetic energies |k + G|^2 / 2, kc the Cartesian k (bohr^-1).
void sphere_miller(const double L[3], const double kfrac[3], double ecut, std::vector<int>& miller,
                   std::vector<double>& kin, double kc[3]);

// Ewald energy of point charges Z at Cartesian positions pos [n][3] in the orthorhombic cell L
// with a uniform neutralising background (the nuclear repulsion V_NN of the total energy).
double ewald_energy(const double L[3], const std::vector<double>& pos, const std::vector<double>& Z);

// Occupations of nk x nb eigenvalues eig [nk][nb] (Ha) with k weights wk [nk] holding nelec
// electrons: 2 sum_k w_k sum_j n_jk = nelec.  sigma > 0: smeared, n = f((e - mu) / sigma) with
// f of kind (FDE_SMEAR_FERMI, FDE_SMEAR_MP first-order Methfessel-Paxton, FDE_SMEAR_GAUSS), mu by
// bisection to |N(mu) - nelec| < 1e-13, and ts = sigma S, S = 2 sum_k w_k sum_j s(x_jk) with s
// the entropy-like term of the same kind (Fermi-Dirac: the Mermin entropy).  sigma <= 0:
// integer occupations of the nelec / 2 lowest bands (one k-point), mu = the highest occupied
// eigenvalue, ts = 0.  Returns false for inconsistent arguments.
bool occupations_host(int nk, int nb, const double* eig, const double* wk, double nelec, double sigma, double* occ,
                      double* mu, double* ts, int kind);

// Monkhorst-Pack mesh q[0] x q[1] x q[2] with offsets shift[3] (nullable: unshifted),
// k_j = (2 r_j - q_j - 1 + shift_j) / (2 q_j), r_j = 1..q_j, reduced to one point per orbit of
// {R k, and -R k if time_reversal} (R over the identity and the sign-flip masks ops[nops]):
// kpts [nk][3] (crystal coordinates, the first member of each orbit in mesh order) and wk [nk] =
// orbit size / mesh size.  False for bad arguments.
bool kmesh_host(const int q[3], const double shift[3], int time_reversal, int nops, const int* ops,
                std::vector<double>& kpts, std::vector<double>& wk);

// Sign-flip operations about the origin (3-bit masks, identity first) mapping the atoms onto
// atoms of equal charge within tol (bohr) modulo the orthorhombic cell L.
void symmetry_ops_host(const double L[3], int natoms, const double* pos, const double* Z, double tol,
                       std::vector<int>& ops);

// Gaussian elimination with partial pivoting on the dense n x n system A x = b (row-major);
// the solution replaces b.  False for a (numerically) singular A.
bool solve_dense(std::vector<double>& A, std::vector<double>& b, int n);

// Pulay (DIIS) coefficients: minimise |sum_i c_i R_i|^2 subject to sum_i c_i = 1, given the
// residual overlaps ov[i][j] = <R_i|R_j> (m x m, row-major).  When the bordered system is
// singular the last residual gets the whole weight (c = e_m) and false is returned.
bool pulay_coefficients(const double* ov, int m, double* coef);

}  // namespace fde
