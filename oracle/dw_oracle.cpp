// Domain-wall fermion operator: plain FP64 CPU oracle.
//
// TEST INFRASTRUCTURE ONLY. This file is the independent reference that the
// GPU path is checked against. Only the tests, the smoke check and the
// benchmark's CPU-baseline leg may load it; the product library never does.
// It shares no source, header, table or helper with the CUDA path.
//
// What it computes (the paper names the "Domain Wall kernel" and its per-site
// work -- spin projection, SU(3) x half spinor, reconstruction, 1320 flop per
// lattice-site update, Sec. 4.3 and Table 3 -- but never writes the operator
// down; the definitions below are the standard domain-wall operator in the
// reading stated next to each function):
//
//   Dhop psi(x,s) = sum_mu [ (1 - g_mu) U_mu(x) psi(x+mu,s)
//                          + (1 + g_mu) U_mu(x-mu)^+ psi(x-mu,s) ]
//   (Dhop^+ flips the sign in front of g_mu.)  A hop that crosses the lattice
//   edge in direction mu picks up the factor bc[mu] (+1 periodic, -1
//   antiperiodic).
//   D_W   = (4 - M5) - 1/2 Dhop
//   K psi_s = P- psi_{s+1} + P+ psi_{s-1}, walls: -mf P- psi_0 at s=Ls-1 and
//             -mf P+ psi_{Ls-1} at s=0          (P+- = (1 +- g5)/2)
//   D     = D_W (b + c K) + (1 - K)               (Shamir: b=1, c=0)
//   D^+   = (b + c K^+) D_W^+ + (1 - K^+)
//
// Everything is written out with full 4x4 spin matrices and 3x3 colour
// matrices in std::complex<double>; there is no half-spinor trick, no
// blocking and no reordering of the sums beyond the definitions above.
//
// Canonical layouts (shared with the boundary, interleaved re/im doubles):
//   fermion complex128 [rhs][x4][s][spin 4][colour 3],
//   gauge   complex128 [x4][mu = x,y,z,t][row 3][col 3],
//   x4 = x + Lx*(y + Ly*(z + Lz*t)); U_mu(x) links x to x+mu.

#include <complex>
#include <cmath>
#include <cstring>
#include <cstdlib>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef std::complex<double> cplx;

namespace {

// Chiral basis: g_k = [[0, i s_k], [-i s_k, 0]] (k = 1..3), g_4 = [[0,1],[1,0]],
// g5 = diag(1,1,-1,-1).  Typed in by hand from the Pauli matrices.
cplx GAM[4][4][4];
double G5[4];

void init_gamma() {
  static bool done = false;
  if (done) return;
  const cplx I(0.0, 1.0), O(0.0, 0.0), E(1.0, 0.0);
  for (int m = 0; m < 4; ++m)
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) GAM[m][a][b] = O;
  // i*sigma_1 = [[0, i], [i, 0]]
  GAM[0][0][3] = I;   GAM[0][1][2] = I;
  GAM[0][2][1] = -I;  GAM[0][3][0] = -I;
  // i*sigma_2 = [[0, 1], [-1, 0]]
  GAM[1][0][3] = E;   GAM[1][1][2] = -E;
  GAM[1][2][1] = -E;  GAM[1][3][0] = E;
  // i*sigma_3 = [[i, 0], [0, -i]]
  GAM[2][0][2] = I;   GAM[2][1][3] = -I;
  GAM[2][2][0] = -I;  GAM[2][3][1] = I;
  // identity blocks
  GAM[3][0][2] = E;   GAM[3][1][3] = E;
  GAM[3][2][0] = E;   GAM[3][3][1] = E;
  G5[0] = 1.0; G5[1] = 1.0; G5[2] = -1.0; G5[3] = -1.0;
  done = true;
}

struct Lat {
  int L[4];
  long V4;
  int Ls;
  int bc[4];
};

void coords(long x4, const Lat &g, int c[4]) {
  for (int m = 0; m < 4; ++m) { c[m] = (int)(x4 % g.L[m]); x4 /= g.L[m]; }
}

long index4(const int c[4], const Lat &g) {
  return c[0] + (long)g.L[0] * (c[1] + (long)g.L[1] * (c[2] + (long)g.L[2] * c[3]));
}

inline const cplx *fermion_at(const cplx *f, const Lat &g, long x4, int s) {
  return f + ((size_t)x4 * g.Ls + s) * 12;
}

// Hopping term at one 4D site x4, all s, for one RHS: adds into out[s][12].
// sgn = +1 gives Dhop, sgn = -1 gives Dhop^+ (sign of g_mu flipped).
void hop_site(cplx *out, const cplx *in, const cplx *U, const Lat &g, long x4, int sgn) {
  int c[4];
  coords(x4, g, c);
  for (int mu = 0; mu < 4; ++mu) {
    // forward neighbour x + mu
    int cf[4] = {c[0], c[1], c[2], c[3]};
    double ff = 1.0;
    cf[mu] += 1;
    if (cf[mu] == g.L[mu]) { cf[mu] = 0; ff = g.bc[mu]; }
    long yf = index4(cf, g);
    // backward neighbour x - mu
    int cb[4] = {c[0], c[1], c[2], c[3]};
    double fb = 1.0;
    cb[mu] -= 1;
    if (cb[mu] < 0) { cb[mu] = g.L[mu] - 1; fb = g.bc[mu]; }
    long yb = index4(cb, g);

    const cplx *Uf = U + ((size_t)x4 * 4 + mu) * 9;  // U_mu(x)
    const cplx *Ub = U + ((size_t)yb * 4 + mu) * 9;  // U_mu(x - mu)

    // spin matrices (1 - sgn g_mu) and (1 + sgn g_mu)
    cplx Pm[4][4], Pp[4][4];
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) {
        cplx d = (a == b) ? cplx(1.0, 0.0) : cplx(0.0, 0.0);
        Pm[a][b] = d - (double)sgn * GAM[mu][a][b];
        Pp[a][b] = d + (double)sgn * GAM[mu][a][b];
      }

    for (int s = 0; s < g.Ls; ++s) {
      const cplx *pf = fermion_at(in, g, yf, s);
      const cplx *pb = fermion_at(in, g, yb, s);
      // colour: U psi and U^+ psi for each spin
      cplx tf[4][3], tb[4][3];
      for (int sp = 0; sp < 4; ++sp)
        for (int r = 0; r < 3; ++r) {
          cplx af(0.0, 0.0), ab(0.0, 0.0);
          for (int k = 0; k < 3; ++k) {
            af += Uf[r * 3 + k] * pf[sp * 3 + k];
            ab += std::conj(Ub[k * 3 + r]) * pb[sp * 3 + k];
          }
          tf[sp][r] = af * ff;
          tb[sp][r] = ab * fb;
        }
      // spin
      cplx *o = out + (size_t)s * 12;
      for (int a = 0; a < 4; ++a)
        for (int r = 0; r < 3; ++r) {
          cplx acc(0.0, 0.0);
          for (int b = 0; b < 4; ++b) acc += Pm[a][b] * tf[b][r] + Pp[a][b] * tb[b][r];
          o[a * 3 + r] += acc;
        }
    }
  }
}

// The 5th-dimension hop K (dag = 0) or K^+ (dag = 1) at one 4D site, all s.
// out[s] = sum_s' K[s][s'] in[s'] (overwrites out).
//   [K psi]_s   = P- psi_{s+1} + P+ psi_{s-1}
//   [K^+ psi]_s = P+ psi_{s+1} + P- psi_{s-1}
// At the walls the neighbour s+1 = Ls is replaced by -mf psi_0 and the
// neighbour s-1 = -1 by -mf psi_{Ls-1}.  P+- = (1 +- g5)/2 is diagonal in the
// chiral basis, so its entries are (1 +- G5[a]) / 2.
void k_site(cplx *out, const cplx *in, int Ls, double mf, int dag) {
  for (int s = 0; s < Ls; ++s) {
    int next = s + 1, prev = s - 1;
    double fn = 1.0, fp = 1.0;
    if (next == Ls) { next = 0; fn = -mf; }
    if (prev < 0) { prev = Ls - 1; fp = -mf; }
    cplx *o = out + (size_t)s * 12;
    const cplx *pn = in + (size_t)next * 12;
    const cplx *pp = in + (size_t)prev * 12;
    for (int a = 0; a < 4; ++a) {
      const double pplus = 0.5 * (1.0 + G5[a]);
      const double pminus = 0.5 * (1.0 - G5[a]);
      const double cn = dag ? pplus : pminus;
      const double cp = dag ? pminus : pplus;
      for (int r = 0; r < 3; ++r)
        o[a * 3 + r] = cn * fn * pn[a * 3 + r] + cp * fp * pp[a * 3 + r];
    }
  }
}

// Diagonal-in-x part and assembly of the domain-wall operator at one 4D site.
// dag = 0:  D psi   = (4 - M5) phi - 1/2 Dhop phi + psi - K psi,  phi = (b + cK) psi,
//           with `phi` the full field (b + cK) psi of this RHS.
// dag = 1:  D^+ psi = b chi + c K^+ chi + psi - K^+ psi,
//           chi = D_W^+ psi = (4 - M5) psi - 1/2 Dhop^+ psi.
void dw_site(cplx *out, const cplx *in, const cplx *phi, const cplx *U, const Lat &g, long x4,
             double M5, double b, double c, double mf, int dag) {
  const int Ls = g.Ls;
  const size_t n = (size_t)Ls * 12;
  std::vector<cplx> hop(n, cplx(0.0, 0.0)), kin(n), chi(n), kchi(n);
  const cplx *psi = fermion_at(in, g, x4, 0);
  if (!dag) {
    hop_site(hop.data(), phi, U, g, x4, +1);
    const cplx *phix = fermion_at(phi, g, x4, 0);
    k_site(kin.data(), psi, Ls, mf, 0);
    for (size_t i = 0; i < n; ++i)
      out[i] = (4.0 - M5) * phix[i] - 0.5 * hop[i] + psi[i] - kin[i];
  } else {
    hop_site(hop.data(), in, U, g, x4, -1);
    for (size_t i = 0; i < n; ++i) chi[i] = (4.0 - M5) * psi[i] - 0.5 * hop[i];
    k_site(kchi.data(), chi.data(), Ls, mf, 1);
    k_site(kin.data(), psi, Ls, mf, 1);
    for (size_t i = 0; i < n; ++i) out[i] = b * chi[i] + c * kchi[i] + psi[i] - kin[i];
  }
}

bool make_lat(Lat &g, const int *dims, int Ls, const int *bc) {
  init_gamma();
  if (!dims || Ls < 1) return false;
  g.V4 = 1;
  for (int m = 0; m < 4; ++m) {
    if (dims[m] < 1) return false;
    g.L[m] = dims[m];
    g.V4 *= dims[m];
    g.bc[m] = bc ? bc[m] : (m == 3 ? -1 : 1);
  }
  g.Ls = Ls;
  return true;
}

}  // namespace

extern "C" {

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

// Dhop (dag = 0) or Dhop^+ (dag = 1), bare hopping sum, no -1/2 and no diagonal.
// sites == NULL: all 4D sites, out is a full canonical field.
// otherwise: out is [rhs][nsites][Ls][12] complex for the listed 4D sites.
int oracle_dhop(double *out, const double *in, const double *U, const int *dims, int Ls,
                int nrhs, const int *bc, int dag, const long *sites, long nsites) {
  Lat g;
  if (!make_lat(g, dims, Ls, bc) || !out || !in || !U || nrhs < 1) return -1;
  const cplx *pin = reinterpret_cast<const cplx *>(in);
  const cplx *pU = reinterpret_cast<const cplx *>(U);
  cplx *pout = reinterpret_cast<cplx *>(out);
  const long ns = sites ? nsites : g.V4;
  const size_t fsz = (size_t)g.V4 * Ls * 12;
  const size_t osz = (size_t)ns * Ls * 12;
  for (int r = 0; r < nrhs; ++r) {
#pragma omp parallel for schedule(static)
    for (long i = 0; i < ns; ++i) {
      long x4 = sites ? sites[i] : i;
      cplx *o = pout + r * osz + (size_t)i * Ls * 12;
      for (int k = 0; k < Ls * 12; ++k) o[k] = 0.0;
      hop_site(o, pin + r * fsz, pU, g, x4, dag ? -1 : 1);
    }
  }
  return 0;
}

// The 5D hop K or K^+ on a full field (5D-local).
int oracle_k(double *out, const double *in, const int *dims, int Ls, int nrhs,
             const double *mf, int dag) {
  Lat g;
  if (!make_lat(g, dims, Ls, nullptr) || !out || !in || !mf) return -1;
  const cplx *pin = reinterpret_cast<const cplx *>(in);
  cplx *pout = reinterpret_cast<cplx *>(out);
  const size_t fsz = (size_t)g.V4 * Ls * 12;
  for (int r = 0; r < nrhs; ++r) {
#pragma omp parallel for schedule(static)
    for (long x4 = 0; x4 < g.V4; ++x4)
      k_site(pout + r * fsz + (size_t)x4 * Ls * 12, pin + r * fsz + (size_t)x4 * Ls * 12, Ls,
             mf[r], dag);
  }
  return 0;
}

// Domain-wall operator D (dag = 0) or D^+ (dag = 1), per-RHS masses mf[nrhs].
// sites as for oracle_dhop.
int oracle_dw(double *out, const double *in, const double *U, const int *dims, int Ls,
              int nrhs, const int *bc, double M5, double b, double c, const double *mf,
              int dag, const long *sites, long nsites) {
  Lat g;
  if (!make_lat(g, dims, Ls, bc) || !out || !in || !U || !mf || nrhs < 1) return -1;
  const cplx *pin = reinterpret_cast<const cplx *>(in);
  const cplx *pU = reinterpret_cast<const cplx *>(U);
  cplx *pout = reinterpret_cast<cplx *>(out);
  const long ns = sites ? nsites : g.V4;
  const size_t fsz = (size_t)g.V4 * Ls * 12;
  const size_t osz = (size_t)ns * Ls * 12;
  std::vector<cplx> phi(dag ? 0 : fsz);
  for (int r = 0; r < nrhs; ++r) {
    const cplx *pr = pin + r * fsz;
    if (!dag) {
      // phi = (b + cK) psi on the whole field (5D-local)
#pragma omp parallel for schedule(static)
      for (long x4 = 0; x4 < g.V4; ++x4) {
        cplx *ph = phi.data() + (size_t)x4 * Ls * 12;
        const cplx *ps = pr + (size_t)x4 * Ls * 12;
        k_site(ph, ps, Ls, mf[r], 0);
        for (int k = 0; k < Ls * 12; ++k) ph[k] = b * ps[k] + c * ph[k];
      }
    }
#pragma omp parallel for schedule(static)
    for (long i = 0; i < ns; ++i) {
      long x4 = sites ? sites[i] : i;
      dw_site(pout + r * osz + (size_t)i * Ls * 12, pr, phi.data(), pU, g, x4, M5, b, c, mf[r],
              dag);
    }
  }
  return 0;
}

// D^+ D on full fields.
int oracle_dwdagdw(double *out, const double *in, const double *U, const int *dims, int Ls,
                   int nrhs, const int *bc, double M5, double b, double c, const double *mf) {
  Lat g;
  if (!make_lat(g, dims, Ls, bc) || !out || !in || !U || !mf || nrhs < 1) return -1;
  const size_t n = (size_t)nrhs * g.V4 * Ls * 24;
  std::vector<double> tmp(n);
  int rc = oracle_dw(tmp.data(), in, U, dims, Ls, nrhs, bc, M5, b, c, mf, 0, nullptr, 0);
  if (rc) return rc;
  return oracle_dw(out, tmp.data(), U, dims, Ls, nrhs, bc, M5, b, c, mf, 1, nullptr, 0);
}

// Textbook conjugate gradient (Hestenes-Stiefel) on A = D^+ D, one RHS at a
// time, FP64 throughout.  x holds the start vector on entry and the solution on
// exit.  Stops when |r_k| / |b| <= tol (recursive residual) or after maxit
// iterations; then recomputes the true residual |b - A x| / |b|.
// iters[r], true_resid[r] are filled per RHS.  Returns 0 when every RHS met tol
// by the true residual, 1 otherwise.
int oracle_cg(double *x, const double *bvec, const double *U, const int *dims, int Ls,
              int nrhs, const int *bc, double M5, double b, double c, const double *mf,
              double tol, int maxit, int *iters, double *true_resid) {
  Lat g;
  if (!make_lat(g, dims, Ls, bc) || !x || !bvec || !U || !mf || nrhs < 1) return -1;
  const size_t n = (size_t)g.V4 * Ls * 24;  // reals per RHS
  std::vector<double> r(n), p(n), Ap(n);
  auto dot = [&](const double *a, const double *bb) {
    // Re <a, b> = sum of products of the real components
    double s = 0.0;
    for (size_t i = 0; i < n; ++i) s += a[i] * bb[i];
    return s;
  };
  int all_ok = 1;
  for (int rh = 0; rh < nrhs; ++rh) {
    double *xr = x + rh * n;
    const double *br = bvec + rh * n;
    const double m = mf[rh];
    oracle_dwdagdw(Ap.data(), xr, U, dims, Ls, 1, bc, M5, b, c, &m);
    for (size_t i = 0; i < n; ++i) { r[i] = br[i] - Ap[i]; p[i] = r[i]; }
    const double bnorm = std::sqrt(dot(br, br));
    double rr = dot(r.data(), r.data());
    int k = 0;
    while (k < maxit && std::sqrt(rr) > tol * bnorm) {
      oracle_dwdagdw(Ap.data(), p.data(), U, dims, Ls, 1, bc, M5, b, c, &m);
      const double alpha = rr / dot(p.data(), Ap.data());
      for (size_t i = 0; i < n; ++i) { xr[i] += alpha * p[i]; r[i] -= alpha * Ap[i]; }
      const double rr_new = dot(r.data(), r.data());
      const double beta = rr_new / rr;
      for (size_t i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
      rr = rr_new;
      ++k;
    }
    oracle_dwdagdw(Ap.data(), xr, U, dims, Ls, 1, bc, M5, b, c, &m);
    double tr = 0.0;
    for (size_t i = 0; i < n; ++i) tr += (br[i] - Ap[i]) * (br[i] - Ap[i]);
    const double res = std::sqrt(tr) / bnorm;
    if (iters) iters[rh] = k;
    if (true_resid) true_resid[rh] = res;
    if (!(res <= tol)) all_ok = 0;
  }
  return all_ok ? 0 : 1;
}

}  // extern "C"
