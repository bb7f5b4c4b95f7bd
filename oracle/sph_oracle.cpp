/*
 * FP64 CPU oracle for the weakly-compressible SPH hot path.
 *
 * TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the CPU
 * baseline of the benchmark may load or call this code.  It shares nothing
 * with the CUDA library: no header, helper, table or constant generator.
 *
 * It is written to be checked against the paper by eye: plain loops, FP64,
 * no blocking or fusion.  Every function cites the passage it follows
 * (arXiv 2207.11328, "Fast, feature-rich weakly-compressible SPH on GPU").
 * Where the paper only cites another work, leaves a symbol undefined or
 * prints a sign or a factor that cannot be right, the reading taken is
 * stated in full beside the formula it affects, with the passage it reads
 * (e.g. the continuity sign of Eq. mass-cont-sph1, the missing m_j of
 * Eq. ns-sph1, the artificial viscosity that Table 1 only names).
 *
 * Scalar type: every formula is a template on the scalar so that the same
 * code runs in double and in forward-mode dual numbers (directional
 * derivatives for the adjoint checks).  Branch decisions (cutoff, artificial
 * viscosity switch, minimum image) are taken on the primal value.
 */
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

extern "C" {

/* Run parameters (oracle-private layout, mirrored by the oracle's Python wrapper). */
typedef struct {
    double dp, h, kernel_radius;   /* influence radius R = kernel_radius*h (Section 2.1, compact support) */
    double rho0, c0, gamma;        /* Cole/Tait equation of state, Section 2.1 */
    int32_t visc_model;            /* 0 artificial (Monaghan), laminar: 1 Morris, 2 Monaghan, 3 Espanol & Revenga */
    int32_t pad0;
    double alpha, nu;              /* artificial-viscosity coefficient / kinematic viscosity */
    double g[3];                   /* body force, fluid only */
    double cfl, dt_fixed;          /* dt_fixed > 0 freezes the time step */
    double origin[3], size[3];     /* domain; periodic axes wrap with period size[axis] */
    uint32_t periodic_mask;        /* bit0 x, bit1 y, bit2 z */
    uint32_t pad1;
    /* model options of Table 1 (0 everywhere = the model above) */
    int32_t kernel_type;           /* 0 Wendland C2, 1 cubic spline, 2 quadratic, 3 Gaussian */
    int32_t formulation;           /* 0 eqs. mass-cont-sph1/ns-sph1, 1 eqs. mass-cont-sph2/ns-sph2 */
    int32_t visc_avg;              /* laminar models: 0 harmonic, 1 arithmetic, 2 geometric mean */
    int32_t ddiff;                 /* density diffusion: 0 none, 1 Molteni & Colagrossi */
    double ddiff_coef;             /* its coefficient xi */
    double zeta;                   /* kinematic bulk viscosity (Espanol & Revenga model) */
} ora_params;

}  // extern "C"

namespace {

const double kPi = 3.14159265358979323846;

/* ------------------------------------------------------------------ */
/* Dual numbers for forward-mode derivatives.                          */
/* ------------------------------------------------------------------ */
struct Dual {
    double v, d;
    Dual() : v(0), d(0) {}
    Dual(double a) : v(a), d(0) {}
    Dual(double a, double b) : v(a), d(b) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) { return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)); }
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
inline Dual sqrt(Dual a) { double s = std::sqrt(a.v); return Dual(s, a.d / (2.0 * s)); }
inline Dual exp(Dual a) { double e = std::exp(a.v); return Dual(e, a.d * e); }

inline double pv(double a) { return a; }
inline double pv(const Dual& a) { return a.v; }
using std::exp;
using std::sqrt;

/* ------------------------------------------------------------------ */
/* Wendland C2 kernel in 3D, support radius 2h (Section 4, kernel      */
/* templates listing: w(q) = (2q+1)(1-q/2)^4, f(q) = (q-2)^3).          */
/* The listing leaves the normalisation coefficients as precomputed    */
/* constants; the unit-integral property of Section 2.1 fixes them:    */
/*   a_W = 21/(16 pi h^3),  F = (1/r) dW/dr  =>  a_F = 105/(128 pi h^5) */
/* ------------------------------------------------------------------ */
template <class T>
T kernel_W(T r, double h) {
    T q = r / h;
    if (pv(q) >= 2.0) return T(0.0);
    T t = T(1.0) - q * 0.5;
    return T(21.0 / (16.0 * kPi * h * h * h)) * t * t * t * t * (q * 2.0 + T(1.0));
}

template <class T>
T kernel_F(T r, double h) {
    T q = r / h;
    if (pv(q) >= 2.0) return T(0.0);
    T qm2 = q - T(2.0);
    return T(105.0 / (128.0 * kPi * h * h * h * h * h)) * qm2 * qm2 * qm2;
}

/* ------------------------------------------------------------------ */
/* The other smoothing kernels of Table 1 and of the kernel-templates   */
/* listing (Section 4), 3D.  Each is W = a_W w(q) with F = (1/r) dW/dr; */
/* a_W follows from the unit integral 4 pi h^3 a_W int w(q) q^2 dq = 1: */
/*  cubic spline  w = 1 - 3/2 q^2 + 3/4 q^3 (q<1), (2-q)^3/4 (q<2)     */
/*                a_W = 1/(pi h^3)                                       */
/*  quadratic     w = (2-q)^2 (q<2),   a_W = 15/(64 pi h^3)             */
/*  Gaussian      w = exp(-q^2) - exp(-Q^2) (q<Q, Q = kernel_radius),   */
/*                a_W = 1/(4 pi h^3 S(Q)),                               */
/*                S(Q) = sqrt(pi)/4 erf(Q) - (Q/2 + Q^3/3) exp(-Q^2)     */
/* ------------------------------------------------------------------ */
double gaussian_S(double Q) {
    return std::sqrt(kPi) / 4.0 * std::erf(Q) - (Q / 2.0 + Q * Q * Q / 3.0) * std::exp(-Q * Q);
}

template <class T>
T kernel_Wk(int type, double Q, T r, double h) {
    const double h3 = h * h * h;
    T q = r / h;
    if (type == 1) {
        if (pv(q) >= 2.0) return T(0.0);
        if (pv(q) < 1.0) return T(1.0 / (kPi * h3)) * (T(1.0) - q * q * 1.5 + q * q * q * 0.75);
        T t = T(2.0) - q;
        return T(1.0 / (kPi * h3)) * t * t * t * 0.25;
    }
    if (type == 2) {
        if (pv(q) >= 2.0) return T(0.0);
        T t = T(2.0) - q;
        return T(15.0 / (64.0 * kPi * h3)) * t * t;
    }
    if (type == 3) {
        if (pv(q) >= Q) return T(0.0);
        return T(1.0 / (4.0 * kPi * h3 * gaussian_S(Q))) * (exp(-(q * q)) - T(std::exp(-Q * Q)));
    }
    return kernel_W(r, h);
}

/* F = (1/r) dW/dr = a_W w'(q) / (h^2 q):
 *  cubic spline  (-3 + 9/4 q) (q<1),  -3/4 (2-q)^2 / q (q<2),  times 1/(pi h^5)
 *  quadratic     (q - 2)/q,  times 15/(32 pi h^5)
 *  Gaussian      -exp(-q^2), times 1/(2 pi h^5 S(Q))   (no smooth cut at Q) */
template <class T>
T kernel_Fk(int type, double Q, T r, double h) {
    const double h5 = h * h * h * h * h;
    T q = r / h;
    if (type == 1) {
        if (pv(q) >= 2.0) return T(0.0);
        if (pv(q) < 1.0) return T(1.0 / (kPi * h5)) * (q * 2.25 - T(3.0));
        T t = T(2.0) - q;
        return T(1.0 / (kPi * h5)) * (t * t * -0.75) / q;
    }
    if (type == 2) {
        if (pv(q) >= 2.0) return T(0.0);
        return T(15.0 / (32.0 * kPi * h5)) * (q - T(2.0)) / q;
    }
    if (type == 3) {
        if (pv(q) >= Q) return T(0.0);
        return -T(1.0 / (2.0 * kPi * h5 * gaussian_S(Q))) * exp(-(q * q));
    }
    return kernel_F(r, h);
}

/* Averaging operator of Table 1 for two positive values. */
template <class T>
T average(int op, T a, T b) {
    if (op == 1) return (a + b) * 0.5;
    if (op == 2) return sqrt(a * b);
    return a * b * 2.0 / (a + b);
}

/* ------------------------------------------------------------------ */
/* Cole equation of state, Section 2.1: P = B((rho/rho0)^gamma - 1),   */
/* B = rho0 c0^2 / gamma.  With delta = rho/rho0 - 1 and integer gamma */
/* the binomial expansion gives P = B*delta*sum_k C(gamma,k) delta^(k-1)*/
/* exactly, without the cancellation of (1+delta)^gamma - 1.           */
/* ------------------------------------------------------------------ */
template <class T>
T eos_pressure(T delta, const ora_params& P) {
    int gam = (int)std::lround(P.gamma);
    double B = P.rho0 * P.c0 * P.c0 / P.gamma;
    T sum(0.0), dpow(1.0);
    double binom = 1.0;  /* C(gam, k) built incrementally */
    for (int k = 1; k <= gam; ++k) {
        binom = binom * (double)(gam - k + 1) / (double)k;
        sum += dpow * binom;
        dpow = dpow * delta;
    }
    return T(B) * delta * sum;
}

bool is_periodic(const ora_params& P, int axis) { return (P.periodic_mask >> axis) & 1u; }

/* Separation x_i - x_j with the minimum-image convention on periodic axes
 * (Table 1 "periodicity in any of X, Y, Z"); the image shift is chosen on
 * the primal value. */
template <class T>
void separation(const ora_params& P, const T* xi, const T* xj, T* d) {
    for (int a = 0; a < 3; ++a) {
        d[a] = xi[a] - xj[a];
        if (is_periodic(P, a)) {
            double L = P.size[a];
            double k = std::nearbyint(pv(d[a]) / L);
            d[a] = d[a] - T(k * L);
        }
    }
}

/* ------------------------------------------------------------------ */
/* Neighbour sets, Section 2.3: all j != i with 0 < r_ij < R.          */
/* Brute force O(N^2), or a simple binning of its own (bins of side    */
/* >= R, 27 bins around each particle, Figure "search radius").        */
/* Output in CSR form, neighbours of each i in increasing index.       */
/* ------------------------------------------------------------------ */
struct Nbrs {
    std::vector<int64_t> off;
    std::vector<int32_t> idx;
};

double radius(const ora_params& P) { return P.kernel_radius * P.h; }

void neighbors_brute(const ora_params& P, int n, const double* x, Nbrs& out) {
    const double R2 = radius(P) * radius(P);
    out.off.assign(n + 1, 0);
    out.idx.clear();
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            double d[3];
            separation(P, x + 3 * i, x + 3 * j, d);
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (r2 > 0.0 && r2 < R2) out.idx.push_back(j);
        }
        out.off[i + 1] = (int64_t)out.idx.size();
    }
}

struct Bins {
    int nb[3];
    double side[3];
    std::vector<int64_t> start;   /* per bin, size nbins+1 */
    std::vector<int32_t> order;   /* particle indices sorted by bin */
    std::vector<int64_t> bin_of;  /* per particle */
};

bool make_bins(const ora_params& P, int n, const double* x, Bins& B) {
    const double R = radius(P);
    for (int a = 0; a < 3; ++a) {
        int k = (int)std::floor(P.size[a] / R);
        if (k < 1) k = 1;
        if (is_periodic(P, a) && k < 3) return false;  /* minimum image needs >= 3 bins */
        B.nb[a] = k;
        B.side[a] = P.size[a] / k;
    }
    const int64_t nbins = (int64_t)B.nb[0] * B.nb[1] * B.nb[2];
    B.bin_of.resize(n);
    std::vector<int64_t> cnt(nbins + 1, 0);
    for (int i = 0; i < n; ++i) {
        int64_t c[3];
        for (int a = 0; a < 3; ++a) {
            double t = (x[3 * i + a] - P.origin[a]) / B.side[a];
            int64_t k = (int64_t)std::floor(t);
            if (is_periodic(P, a)) {
                k %= B.nb[a];
                if (k < 0) k += B.nb[a];
            } else {
                k = std::min<int64_t>(std::max<int64_t>(k, 0), B.nb[a] - 1);
            }
            c[a] = k;
        }
        B.bin_of[i] = c[0] + B.nb[0] * (c[1] + B.nb[1] * c[2]);
        cnt[B.bin_of[i] + 1]++;
    }
    for (int64_t b = 0; b < nbins; ++b) cnt[b + 1] += cnt[b];
    B.start = cnt;
    B.order.resize(n);
    std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
    for (int i = 0; i < n; ++i) B.order[fill[B.bin_of[i]]++] = i;
    return true;
}

/* Neighbours of particle i from the bins, increasing index. */
void neighbors_of(const ora_params& P, const double* x, const Bins& B, int i,
                  std::vector<int32_t>& nb) {
    const double R2 = radius(P) * radius(P);
    nb.clear();
    int64_t b = B.bin_of[i];
    int c[3] = {(int)(b % B.nb[0]), (int)((b / B.nb[0]) % B.nb[1]), (int)(b / ((int64_t)B.nb[0] * B.nb[1]))};
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int cc[3] = {c[0] + dx, c[1] + dy, c[2] + dz};
                bool skip = false;
                for (int a = 0; a < 3; ++a) {
                    if (is_periodic(P, a)) {
                        cc[a] = (cc[a] % B.nb[a] + B.nb[a]) % B.nb[a];
                    } else if (cc[a] < 0 || cc[a] >= B.nb[a]) {
                        skip = true;
                    }
                }
                if (skip) continue;
                int64_t bb = cc[0] + (int64_t)B.nb[0] * (cc[1] + (int64_t)B.nb[1] * cc[2]);
                for (int64_t s = B.start[bb]; s < B.start[bb + 1]; ++s) {
                    int j = B.order[s];
                    if (j == i) continue;
                    double d[3];
                    separation(P, x + 3 * i, x + 3 * j, d);
                    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                    if (r2 > 0.0 && r2 < R2) nb.push_back(j);
                }
            }
    std::sort(nb.begin(), nb.end());
}

void neighbors_grid(const ora_params& P, int n, const double* x, Nbrs& out) {
    Bins B;
    if (!make_bins(P, n, x, B)) {
        neighbors_brute(P, n, x, out);
        return;
    }
    out.off.assign(n + 1, 0);
    out.idx.clear();
    std::vector<int32_t> nb;
    for (int i = 0; i < n; ++i) {
        neighbors_of(P, x, B, i, nb);
        out.idx.insert(out.idx.end(), nb.begin(), nb.end());
        out.off[i + 1] = (int64_t)out.idx.size();
    }
}

/* ------------------------------------------------------------------ */
/* Time derivatives of one particle (Section 2.1, golden-rule form,    */
/* equations mass-cont-sph1 and ns-sph1 with the readings below).      */
/*                                                                      */
/*  drho_i/dt = + sum_j m_j (u_i - u_j) . x_ij F_ij           (C1)      */
/*  du_i/dt   = - sum_j m_j (P_i/rho_i^2 + P_j/rho_j^2 + Pi_ij) x_ij F_ij */
/*              + sum_j 4 nu m_j/(rho_i+rho_j) F_ij (u_i - u_j)   (C2,C3)*/
/*              + g                                                     */
/*  Pi_ij = -alpha h c0 mu_ij / rhobar_ij  if u_ij.x_ij < 0, else 0    */
/*  mu_ij = u_ij.x_ij / (r^2 + 0.01 h^2),  rhobar = (rho_i+rho_j)/2 (C4)*/
/*  Dynamic boundary particles (C5): velocity zero, positions fixed,   */
/*  continuity and EOS as fluid, no momentum equation.                 */
/*                                                                      */
/* Model options (Table 1; Section 3, viscous-term specialisations):   */
/*  formulation 2 (eqs. mass-cont-sph2, ns-sph2; readings C1, C2):     */
/*    drho_i/dt = + sum_j (rho_i/rho_j) m_j u_ij.x_ij F_ij              */
/*    pressure    - sum_j m_j ((P_i + P_j)/(rho_i rho_j) + Pi_ij) x_ij F_ij */
/*  laminar viscous models, omega_ij = m_j/(rho_i rho_j), mubar_ij the */
/*  average of mu = rho nu (zetabar of rho zeta):                       */
/*    Morris    + sum_j omega 2 mubar F u_ij                             */
/*    Monaghan  + K sum_j omega 2 mubar F (x.u/x.x) x_ij, K = 5 (C14)    */
/*    Espanol & Revenga + sum_j omega F ((5/3 mubar - zetabar) u_ij      */
/*                         + 5 (mubar/3 + zetabar) (x.u/x.x) x_ij)       */
/*  density diffusion, Molteni & Colagrossi (reading D1): fluid pairs  */
/*    + xi h c0 sum_j psi_ij . grad_i W_ij m_j/rho_j,                   */
/*    psi_ij = 2 (rho_j - rho_i) x_ji / |x_ij|^2, grad_i W_ij = x_ij F_ij */
/*    = + 2 xi h c0 sum_j (rho_i - rho_j) F_ij m_j/rho_j                 */
/* ------------------------------------------------------------------ */
template <class T>
struct State {
    std::vector<T> x, u, delta;  /* 3n, 3n, n */
};

/* mag (nullable): receives the summed magnitudes of the pair terms,
 * mag[0] = |g| + sum_j |momentum term_ij|, mag[1] = sum_j |continuity term_ij|
 * (the scale of the cancellation in each sum; used to state FP32 error bounds). */
template <class T>
void particle_rhs(const ora_params& P, int i, const T* x, const T* u, const T* delta,
                  const double* m, const uint8_t* type, T alpha, const T* rho, const T* phat,
                  const int32_t* nb, int64_t nnb, T* a_out, T* drho_out, double* mag = nullptr) {
    double mag_a = 0.0, mag_d = 0.0;
    const double h = P.h;
    const bool fluid_i = type[i] == 0;
    const bool form2 = P.formulation == 1;
    T ui[3];
    for (int c = 0; c < 3; ++c) ui[c] = fluid_i ? u[3 * i + c] : T(0.0);
    T drho(0.0), a[3] = {T(0.0), T(0.0), T(0.0)};
    for (int64_t k = 0; k < nnb; ++k) {
        const int j = nb[k];
        T d[3];
        separation(P, x + 3 * i, x + 3 * j, d);
        T r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        if (!(pv(r2) > 0.0)) continue;
        T r = sqrt(r2);
        T F = kernel_Fk(P.kernel_type, P.kernel_radius, r, h);
        const bool fluid_j = type[j] == 0;
        T uij[3];
        for (int c = 0; c < 3; ++c) uij[c] = ui[c] - (fluid_j ? u[3 * j + c] : T(0.0));
        T udotx = uij[0] * d[0] + uij[1] * d[1] + uij[2] * d[2];
        T mc = form2 ? T(m[j]) * rho[i] / rho[j] : T(m[j]);
        drho += mc * udotx * F;
        if (mag) mag_d += std::fabs(pv(mc * udotx * F));
        if (P.ddiff == 1 && fluid_i && fluid_j) {
            T dd = T(2.0 * P.ddiff_coef * h * P.c0) * (rho[i] - rho[j]) * F * T(m[j]) / rho[j];
            drho += dd;
            if (mag) mag_d += std::fabs(pv(dd));
        }
        if (!fluid_i) continue;
        T bracket = form2 ? (eos_pressure(delta[i], P) + eos_pressure(delta[j], P)) / (rho[i] * rho[j])
                          : phat[i] + phat[j];
        if (P.visc_model == 0 && pv(udotx) < 0.0) {
            T mu = udotx / (r2 + T(0.01 * h * h));
            T rhobar = (rho[i] + rho[j]) * 0.5;
            bracket += -(alpha * (h * P.c0)) * mu / rhobar;
        }
        T coef = T(m[j]) * bracket * F;
        for (int c = 0; c < 3; ++c) a[c] -= coef * d[c];
        if (mag) mag_a += std::fabs(pv(coef)) * std::sqrt(pv(r2));
        if (P.visc_model >= 1) {
            T omega = T(m[j]) / (rho[i] * rho[j]);
            T mubar = average(P.visc_avg, rho[i], rho[j]) * P.nu;
            T lu(0.0), lx(0.0);  /* a += lu * u_ij + lx * x_ij */
            if (P.visc_model == 1) {
                lu = omega * 2.0 * mubar * F;
            } else if (P.visc_model == 2) {
                lx = omega * 2.0 * mubar * F * udotx / r2 * 5.0;
            } else {
                T zetabar = average(P.visc_avg, rho[i], rho[j]) * P.zeta;
                lu = omega * F * (mubar * (5.0 / 3.0) - zetabar);
                lx = omega * F * (mubar / 3.0 + zetabar) * 5.0 * udotx / r2;
            }
            for (int c = 0; c < 3; ++c) a[c] += lu * uij[c] + lx * d[c];
            if (mag)
                mag_a += std::fabs(pv(lu)) * std::sqrt(pv(uij[0] * uij[0] + uij[1] * uij[1] + uij[2] * uij[2])) +
                         std::fabs(pv(lx)) * std::sqrt(pv(r2));
        }
    }
    if (mag) {
        mag[0] = mag_a + (fluid_i ? std::sqrt(P.g[0] * P.g[0] + P.g[1] * P.g[1] + P.g[2] * P.g[2]) : 0.0);
        mag[1] = mag_d;
    }
    if (fluid_i) {
        for (int c = 0; c < 3; ++c) a_out[c] = a[c] + T(P.g[c]);
    } else {
        for (int c = 0; c < 3; ++c) a_out[c] = T(0.0);
    }
    *drho_out = drho;
}

template <class T>
void rhs_all(const ora_params& P, int n, const T* x, const T* u, const T* delta, const double* m,
             const uint8_t* type, T alpha, const Nbrs& N, T* a, T* drho) {
    std::vector<T> rho(n), phat(n);
    for (int i = 0; i < n; ++i) {
        rho[i] = T(P.rho0) * (T(1.0) + delta[i]);
        phat[i] = eos_pressure(delta[i], P) / (rho[i] * rho[i]);
    }
    for (int i = 0; i < n; ++i)
        particle_rhs(P, i, x, u, delta, m, type, alpha, rho.data(), phat.data(),
                     N.idx.data() + N.off[i], N.off[i + 1] - N.off[i], a + 3 * i, drho + i);
}

/* CFL time step (reading C7): dt = min(cfl * min(min_i sqrt(h/|a_i|) over
 * fluid, h/c0), 0.125 h^2/nu for laminar viscosity).  Table 1 "adaptive
 * time-stepping"; Section "The GPU in GPUSPH": the minimum is a reduction over
 * particles.  The viscous limit carries its own coefficient, not the CFL
 * factor: the laminar term's fastest mode on the lattice (neighbours of odd
 * parity moving against the particle) decays at lambda ~ 7 nu/h^2 at
 * h = 1.3 dp, and the two-stage predictor-corrector is stable for a real
 * negative eigenvalue only while lambda dt <= 2; 0.125 h^2/nu (the explicit
 * viscous-diffusion limit usual for SPH) keeps lambda dt below 1. */
constexpr double kViscousDtCoef = 0.125;

double cfl_dt(const ora_params& P, int n, const double* a, const uint8_t* type) {
    double amax2 = 0.0;
    for (int i = 0; i < n; ++i) {
        if (type[i] != 0) continue;
        double s = a[3 * i] * a[3 * i] + a[3 * i + 1] * a[3 * i + 1] + a[3 * i + 2] * a[3 * i + 2];
        amax2 = std::max(amax2, s);
    }
    double dt = P.h / P.c0;
    if (amax2 > 0.0) dt = std::min(dt, std::sqrt(P.h / std::sqrt(amax2)));
    dt *= P.cfl;
    if (P.visc_model >= 1 && P.nu > 0.0) dt = std::min(dt, kViscousDtCoef * P.h * P.h / P.nu);
    return dt;
}

void wrap_positions(const ora_params& P, int n, double* x) {
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a)
            if (is_periodic(P, a)) {
                double L = P.size[a];
                double t = x[3 * i + a] - P.origin[a];
                t -= L * std::floor(t / L);
                if (t >= L) t -= L;
                x[3 * i + a] = P.origin[a] + t;
            }
}

/* One predictor-corrector step (reading C6; Section "Code structure": the
 * integrator runs forces and integration twice per step, with dt/2 and dt).
 *   forces at n ->  u* = u + dt/2 a,  delta* = delta + dt/2 ddelta,  x* = x + dt/2 u
 *   forces at *  (same neighbour sets)
 *   u' = u + dt a*,  delta' = delta + dt ddelta*,  x' = x + dt (u + u')/2
 * Boundary particles integrate delta only. */
template <class T>
void pc_step(const ora_params& P, int n, T* x, T* u, T* delta, const double* m,
             const uint8_t* type, T alpha, double dt, const Nbrs& N, std::vector<T>& a,
             std::vector<T>& drho) {
    a.assign(3 * n, T(0.0));
    drho.assign(n, T(0.0));
    rhs_all(P, n, x, u, delta, m, type, alpha, N, a.data(), drho.data());
    std::vector<T> xs(x, x + 3 * n), us(u, u + 3 * n), ds(delta, delta + n);
    const double rho0 = P.rho0;
    for (int i = 0; i < n; ++i) {
        ds[i] = delta[i] + T(0.5 * dt / rho0) * drho[i];
        if (type[i] != 0) continue;
        for (int c = 0; c < 3; ++c) {
            us[3 * i + c] = u[3 * i + c] + T(0.5 * dt) * a[3 * i + c];
            xs[3 * i + c] = x[3 * i + c] + T(0.5 * dt) * u[3 * i + c];
        }
    }
    rhs_all(P, n, xs.data(), us.data(), ds.data(), m, type, alpha, N, a.data(), drho.data());
    for (int i = 0; i < n; ++i) {
        delta[i] = delta[i] + T(dt / rho0) * drho[i];
        if (type[i] != 0) continue;
        for (int c = 0; c < 3; ++c) {
            T un = u[3 * i + c] + T(dt) * a[3 * i + c];
            x[3 * i + c] = x[3 * i + c] + T(0.5 * dt) * (u[3 * i + c] + un);
            u[3 * i + c] = un;
        }
    }
}

void primal_positions(const std::vector<Dual>& x, std::vector<double>& out) {
    out.resize(x.size());
    for (size_t k = 0; k < x.size(); ++k) out[k] = x[k].v;
}
void primal_positions(const std::vector<double>& x, std::vector<double>& out) { out = x; }

template <class T>
void wrap_T(const ora_params& P, int n, std::vector<T>& x) {
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a)
            if (is_periodic(P, a)) {
                double L = P.size[a];
                double t = pv(x[3 * i + a]) - P.origin[a];
                double k = std::floor(t / L);
                x[3 * i + a] = x[3 * i + a] - T(k * L);
            }
}

}  // namespace

/* ==================================================================== */
/* C entry points                                                        */
/* ==================================================================== */
extern "C" {

double ora_kernel_W(double r, double h) { return kernel_W<double>(r, h); }
double ora_kernel_F(double r, double h) { return kernel_F<double>(r, h); }
/* Any kernel of Table 1: type as ora_params.kernel_type, Q = kernel_radius (Gaussian cut). */
double ora_kernel_Wk(int type, double Q, double r, double h) { return kernel_Wk<double>(type, Q, r, h); }
double ora_kernel_Fk(int type, double Q, double r, double h) { return kernel_Fk<double>(type, Q, r, h); }

double ora_eos(const ora_params* P, double delta) { return eos_pressure<double>(delta, *P); }

/* Neighbour sets in CSR form.  off has n+1 entries; idx has room for cap
 * entries.  Returns the total number of entries, or -needed when cap is
 * too small (nothing written to idx), or -1 on bad arguments. */
int64_t ora_neighbors(const ora_params* P, int n, const double* x, int brute, int64_t cap,
                      int64_t* off, int32_t* idx) {
    if (!P || n < 0) return -1;
    Nbrs N;
    if (brute) neighbors_brute(*P, n, x, N);
    else neighbors_grid(*P, n, x, N);
    int64_t tot = (int64_t)N.idx.size();
    std::memcpy(off, N.off.data(), sizeof(int64_t) * (n + 1));
    if (tot > cap) return -tot;
    if (tot) std::memcpy(idx, N.idx.data(), sizeof(int32_t) * tot);
    return tot;
}

/* Neighbour sets of a sample of particles only (indices sidx[0..ns)), searched
 * among all n particles with the same binning as ora_neighbors (Section 2.3:
 * candidates in the neighbouring cells, reading C9: 0 < r < R).  CSR output:
 * off[0..ns], idx[...] (cap entries at most; returns the total, negated when it
 * exceeds cap). */
int64_t ora_neighbors_sample(const ora_params* P, int n, const double* x, int ns, const int32_t* sidx, int64_t cap,
                             int64_t* off, int32_t* idx) {
    if (!P || n < 0 || ns < 0) return -1;
    Bins B;
    const bool have_bins = make_bins(*P, n, x, B);
    const double R2 = radius(*P) * radius(*P);
    std::vector<int32_t> nb;
    int64_t tot = 0;
    off[0] = 0;
    for (int s = 0; s < ns; ++s) {
        const int i = sidx[s];
        if (have_bins) {
            neighbors_of(*P, x, B, i, nb);
        } else {
            nb.clear();
            for (int j = 0; j < n; ++j) {
                if (j == i) continue;
                double d[3];
                separation(*P, x + 3 * i, x + 3 * j, d);
                double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                if (r2 > 0.0 && r2 < R2) nb.push_back(j);
            }
        }
        for (size_t k = 0; k < nb.size(); ++k) {
            if (tot + (int64_t)k < cap) idx[tot + (int64_t)k] = nb[k];
        }
        tot += (int64_t)nb.size();
        off[s + 1] = tot;
    }
    return tot > cap ? -tot : tot;
}

/* Time derivatives of all particles at the given state.  a: n*3, drho: n,
 * mag: n*2 summed term magnitudes (nullable, see particle_rhs). */
int ora_rhs(const ora_params* P, int n, const double* x, const double* u, const double* delta,
            const double* m, const uint8_t* type, double* a, double* drho, double* mag) {
    if (!P || n < 0) return -1;
    Nbrs N;
    neighbors_grid(*P, n, x, N);
    rhs_all<double>(*P, n, x, u, delta, m, type, P->alpha, N, a, drho);
    if (mag) {
        std::vector<double> rho(n), phat(n), at(3);
        for (int i = 0; i < n; ++i) {
            rho[i] = P->rho0 * (1.0 + delta[i]);
            phat[i] = eos_pressure<double>(delta[i], *P) / (rho[i] * rho[i]);
        }
        double dr;
        for (int i = 0; i < n; ++i)
            particle_rhs<double>(*P, i, x, u, delta, m, type, P->alpha, rho.data(), phat.data(),
                                 N.idx.data() + N.off[i], N.off[i + 1] - N.off[i], at.data(), &dr, mag + 2 * i);
    }
    return 0;
}

/* Time derivatives for a sample of particles only (indices sidx[0..ns)),
 * with neighbours searched among all n particles. */
int ora_rhs_sample(const ora_params* P, int n, const double* x, const double* u,
                   const double* delta, const double* m, const uint8_t* type, int ns,
                   const int32_t* sidx, double* a, double* drho, int32_t* nnb, double* mag) {
    if (!P || n < 0 || ns < 0) return -1;
    Bins B;
    std::vector<int32_t> nb;
    std::vector<double> rho(n), phat(n);
    for (int i = 0; i < n; ++i) {
        rho[i] = P->rho0 * (1.0 + delta[i]);
        phat[i] = eos_pressure<double>(delta[i], *P) / (rho[i] * rho[i]);
    }
    const bool have_bins = make_bins(*P, n, x, B);
    const double R2 = radius(*P) * radius(*P);
    for (int s = 0; s < ns; ++s) {
        int i = sidx[s];
        if (have_bins) {
            neighbors_of(*P, x, B, i, nb);
        } else {
            nb.clear();
            for (int j = 0; j < n; ++j) {
                if (j == i) continue;
                double d[3];
                separation(*P, x + 3 * i, x + 3 * j, d);
                double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                if (r2 > 0.0 && r2 < R2) nb.push_back(j);
            }
        }
        if (nnb) nnb[s] = (int32_t)nb.size();
        particle_rhs<double>(*P, i, x, u, delta, m, type, P->alpha, rho.data(), phat.data(),
                             nb.data(), (int64_t)nb.size(), a + 3 * s, drho + s, mag ? mag + 2 * s : nullptr);
    }
    return 0;
}

double ora_cfl_dt(const ora_params* P, int n, const double* a, const uint8_t* type) {
    return cfl_dt(*P, n, a, type);
}

/* nsteps predictor-corrector steps in place.  Neighbour sets are rebuilt at
 * the start of every step (reading C8).  dt: if P->dt_fixed > 0 it is used
 * for every step; otherwise *dt_io <= 0 asks for dt0 from one forces call on
 * the initial state, and after each step *dt_io holds the CFL dt computed
 * from the corrector-stage accelerations (reading C7).  Positions on periodic
 * axes are wrapped into the domain after each step.  dts (nullable, nsteps
 * entries) receives the dt used by each step. */
int ora_step(const ora_params* P, int n, double* x, double* u, double* delta, const double* m,
             const uint8_t* type, int nsteps, double* dt_io, double* dts) {
    if (!P || n < 0) return -1;
    std::vector<double> a, drho;
    double dt = P->dt_fixed > 0 ? P->dt_fixed : *dt_io;
    if (!(dt > 0)) {
        Nbrs N;
        neighbors_grid(*P, n, x, N);
        a.assign(3 * n, 0.0);
        drho.assign(n, 0.0);
        rhs_all<double>(*P, n, x, u, delta, m, type, P->alpha, N, a.data(), drho.data());
        dt = cfl_dt(*P, n, a.data(), type);
    }
    for (int s = 0; s < nsteps; ++s) {
        Nbrs N;
        neighbors_grid(*P, n, x, N);
        pc_step<double>(*P, n, x, u, delta, m, type, P->alpha, dt, N, a, drho);
        wrap_positions(*P, n, x);
        if (dts) dts[s] = dt;
        if (!(P->dt_fixed > 0)) dt = cfl_dt(*P, n, a.data(), type);
    }
    *dt_io = dt;
    return 0;
}

/* Total energy: kinetic + internal (e(rho) = integral of P/rho^2 drho,
 * B[rho^(g-1)/((g-1) rho0^g) + 1/rho]) + potential -m g.x of the fluid. */
double ora_energy(const ora_params* P, int n, const double* x, const double* u,
                  const double* delta, const double* m, const uint8_t* type) {
    const double B = P->rho0 * P->c0 * P->c0 / P->gamma;
    const double gm = P->gamma;
    double E = 0.0;
    for (int i = 0; i < n; ++i) {
        double rho = P->rho0 * (1.0 + delta[i]);
        E += m[i] * B * (std::pow(rho, gm - 1.0) / ((gm - 1.0) * std::pow(P->rho0, gm)) + 1.0 / rho);
        if (type[i] != 0) continue;
        E += 0.5 * m[i] * (u[3 * i] * u[3 * i] + u[3 * i + 1] * u[3 * i + 1] + u[3 * i + 2] * u[3 * i + 2]);
        E -= m[i] * (P->g[0] * x[3 * i] + P->g[1] * x[3 * i + 1] + P->g[2] * x[3 * i + 2]);
    }
    return E;
}

/* Loss of the differentiable run and its directional derivative.
 *   L = (1/N_f) sum_{fluid i} |x_i(T) - target_i|^2   (minimum image)
 * after T predictor-corrector steps with the frozen dt, from initial state
 * (x0, u0 + eps*0, delta0), artificial-viscosity coefficient alpha.
 * Forward-mode dual numbers carry the tangent (du0, dalpha); neighbour sets
 * are recomputed from the primal positions at every step.  Returns L in
 * *L and the directional derivative dL[du0, dalpha] in *dL. */
int ora_loss_jvp(const ora_params* P, int n, const double* x0, const double* u0,
                 const double* delta0, const double* m, const uint8_t* type, int T, double dt,
                 const double* target, const double* du0, double dalpha, double* L, double* dL) {
    if (!P || n < 0) return -1;
    std::vector<Dual> x(3 * n), u(3 * n), d(n);
    for (int k = 0; k < 3 * n; ++k) {
        x[k] = Dual(x0[k], 0.0);
        u[k] = Dual(u0[k], du0 ? du0[k] : 0.0);
    }
    for (int i = 0; i < n; ++i) d[i] = Dual(delta0[i], 0.0);
    Dual alpha(P->alpha, dalpha);
    std::vector<Dual> a, drho;
    std::vector<double> xp;
    for (int s = 0; s < T; ++s) {
        primal_positions(x, xp);
        Nbrs N;
        neighbors_grid(*P, n, xp.data(), N);
        pc_step<Dual>(*P, n, x.data(), u.data(), d.data(), m, type, alpha, dt, N, a, drho);
        wrap_T(*P, n, x);
    }
    Dual acc(0.0);
    int nf = 0;
    for (int i = 0; i < n; ++i) {
        if (type[i] != 0) continue;
        ++nf;
        Dual dd[3];
        for (int c = 0; c < 3; ++c) {
            dd[c] = x[3 * i + c] - Dual(target[3 * i + c]);
            if (is_periodic(*P, c)) {
                double Lc = P->size[c];
                dd[c] = dd[c] - Dual(Lc * std::nearbyint(dd[c].v / Lc));
            }
        }
        acc += dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2];
    }
    Dual res = acc / Dual((double)(nf > 0 ? nf : 1));
    *L = res.v;
    *dL = res.d;
    return 0;
}

}  // extern "C"
