/*
 * FP64 CPU oracle for one energy+force evaluation of an ANI-2x-shaped
 * neural-network potential.
 *
 * TEST INFRASTRUCTURE ONLY. This file is compiled into liboracle.so and is
 * called by the tests, by the package's smoke check and by the benchmark's
 * CPU-baseline leg. The product library never links, loads or calls it, and
 * it shares no code, header, table or constant generator with the CUDA path.
 *
 * What it computes (paper, section "OpenMM-ML": the ANI-2x potential over the
 * seven elements H, C, N, O, S, F, Cl; section "Optimization Through NNPOps":
 * the bottleneck operations are the atom-centered symmetry functions and the
 * neighbor list; section "PyTorch Model Support": forces are the negative
 * gradient of the energy obtained by backpropagation; section "Performance
 * of MLPs": one net per element, per-atom outputs summed to the energy).
 * The paper does not print the symmetry functions; they are the published
 * ANI (modified Behler-Parrinello) atomic environment vector, restated here
 * from its mathematics:
 *
 *   fc(r; R)  = 0.5 cos(pi r / R) + 0.5 for r < R, else 0
 *   radial    G_i[16 s_j + k]        += 0.25 exp(-eta_R (r_ij - R_k)^2) fc(r_ij; Rc_R)
 *   angular   G_i[112 + 32 p + 8 a + z] += 2 ((1 + cos(theta' - Z_z)) / 2)^zeta
 *                                            * exp(-eta_A ((r_ij + r_ik)/2 - A_a)^2)
 *                                            * fc(r_ij; Rc_A) fc(r_ik; Rc_A)
 *             over unordered neighbor pairs j < k (both within Rc_A),
 *             theta' = acos(0.95 cos theta_ijk), p = index of the unordered
 *             species pair (s_j, s_k) in the row-major upper triangle.
 *   network   e_i = w4 . celu(W3 celu(W2 celu(W1 G_i + b1) + b2) + b3) + b4
 *             with the weights of atom i's element, celu alpha = 0.1.
 *   ensemble  with K nets per element (ANI-2x has eight), e_i is the mean of
 *             the K nets' outputs (section "Performance of MLPs").
 *   energy    E = sum_i e_i;  forces F = -dE/dr (chain rule written out).
 *
 * Hyper-parameters: Rc_R = 5.1 A, 16 radial shifts R_k = linspace(0.8, 4.9),
 * eta_R = 19.7; Rc_A = 3.5 A, A_a = 0.8 + a (3.5 - 0.8)/4 (a = 0..3),
 * Z_z = (2 z + 1) pi / 16 (z = 0..7), eta_A = 12.5, zeta = 14.1; AEV length
 * 7*16 + 28*4*8 = 1008; network 1008-256-192-160-1.
 *
 * Boundary: open, or orthorhombic periodic with the minimum-image convention
 * (nearest-integer rounding of d / L per axis).
 *
 * Pins: every function here is checked by tests against closed forms,
 * library routines, invariants and central finite differences; the whole-path
 * value for random-init weights has no published number.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define NSP 7
#define NRSHIFT 16
#define NASHIFT 4
#define NZSHIFT 8
#define NPAIRS 28
#define RAD_LEN (NSP * NRSHIFT)                     /* 112 */
#define ANG_LEN (NPAIRS * NASHIFT * NZSHIFT)        /* 896 */
#define AEV_LEN (RAD_LEN + ANG_LEN)                 /* 1008 */
#define H1 256
#define H2 192
#define H3 160

static const double RC_RAD = 5.1, ETA_RAD = 19.7;
static const double RC_ANG = 3.5, ETA_ANG = 12.5, ZETA = 14.1;
static const double CELU_ALPHA = 0.1;

/* Per-element weights; every array holds the 7 elements back to back.
 * W1[7][256][1008] b1[7][256] W2[7][192][256] b2[7][192]
 * W3[7][160][192] b3[7][160] W4[7][160] b4[7]   (row = output unit) */
typedef struct {
    const double *W1, *b1, *W2, *b2, *W3, *b3, *W4, *b4;
    int nets; /* ensemble size K; each array holds K nets back to back (0 reads as 1) */
} oracle_weights;

/* ------------------------------------------------------------ AEV pieces */

static double radial_shift(int k) { return 0.8 + k * (4.9 - 0.8) / 15.0; }
static double angular_shift(int a) { return 0.8 + a * (3.5 - 0.8) / 4.0; }
static double section_shift(int z) { return (2.0 * z + 1.0) * M_PI / 16.0; }

/* Cosine cutoff fc(r; R). */
double oracle_cutoff(double r, double rc)
{
    return r < rc ? 0.5 * cos(M_PI * r / rc) + 0.5 : 0.0;
}

/* d fc / d r. */
double oracle_cutoff_deriv(double r, double rc)
{
    return r < rc ? -0.5 * M_PI / rc * sin(M_PI * r / rc) : 0.0;
}

/* CELU with alpha = 0.1: max(0, x) + min(0, alpha (exp(x / alpha) - 1)). */
double oracle_celu(double x)
{
    double neg = CELU_ALPHA * (exp(x / CELU_ALPHA) - 1.0);
    return (x > 0.0 ? x : 0.0) + (neg < 0.0 ? neg : 0.0);
}

/* d celu / d x: 1 for x > 0, exp(x / alpha) otherwise. */
double oracle_celu_deriv(double x)
{
    return x > 0.0 ? 1.0 : exp(x / CELU_ALPHA);
}

/* Index of the unordered species pair (a, b) in the row-major upper
 * triangle of the 7 x 7 species matrix: (0,0)=0 ... (0,6)=6, (1,1)=7 ... */
int oracle_pair_index(int a, int b)
{
    if (a > b) { int t = a; a = b; b = t; }
    int idx = 0;
    for (int r = 0; r < a; ++r) idx += NSP - r;
    return idx + (b - a);
}

/* Displacement d = x_j - x_i, minimum image when cell != NULL. */
static void displacement(const double *xi, const double *xj, const double *cell, double d[3])
{
    for (int c = 0; c < 3; ++c) {
        d[c] = xj[c] - xi[c];
        if (cell) d[c] -= cell[c] * nearbyint(d[c] / cell[c]);
    }
}

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* Brute-force O(N^2) neighbor search: every ordered pair (i, j), j != i,
 * with |d_ij|^2 < rc^2, listed i-major then j ascending. band[p] = 1 marks
 * pairs with | |d|^2 - rc^2 | < 1e-5 rc^2, whose membership a finite-precision
 * search may decide either way. Returns the number of pairs; writes at most
 * cap of them. */
long oracle_neighbors(int n, const double *xyz, const double *cell, double rc,
                      long cap, int *pairs, unsigned char *band)
{
    long cnt = 0;
    double rc2 = rc * rc;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            double d[3];
            displacement(xyz + 3 * i, xyz + 3 * j, cell, d);
            double r2 = dot3(d, d);
            int in = r2 < rc2;
            int near = fabs(r2 - rc2) < 1e-5 * rc2;
            if (in || near) {
                if (cnt < cap) {
                    pairs[2 * cnt] = i;
                    pairs[2 * cnt + 1] = j;
                    if (band) band[cnt] = (unsigned char)(near ? (in ? 1 : 2) : 0);
                }
                ++cnt;
            }
        }
    return cnt;
}

/* Neighbors of atom i within rc (brute force), ascending j. */
static int neighbors_of(int i, int n, const double *xyz, const double *cell, double rc, int *out)
{
    int m = 0;
    for (int j = 0; j < n; ++j) {
        if (j == i) continue;
        double d[3];
        displacement(xyz + 3 * i, xyz + 3 * j, cell, d);
        if (dot3(d, d) < rc * rc) out[m++] = j;
    }
    return m;
}

/* AEV of one atom i: G[1008]. */
static void aev_atom(int i, int n, const int *species, const double *xyz, const double *cell,
                     int *nb, double *G)
{
    memset(G, 0, sizeof(double) * AEV_LEN);
    int m = neighbors_of(i, n, xyz, cell, RC_RAD, nb);
    /* radial */
    for (int q = 0; q < m; ++q) {
        int j = nb[q];
        double d[3];
        displacement(xyz + 3 * i, xyz + 3 * j, cell, d);
        double r = sqrt(dot3(d, d));
        double fc = oracle_cutoff(r, RC_RAD);
        for (int k = 0; k < NRSHIFT; ++k) {
            double t = r - radial_shift(k);
            G[NRSHIFT * species[j] + k] += 0.25 * exp(-ETA_RAD * t * t) * fc;
        }
    }
    /* angular: unordered pairs j < k of neighbors within RC_ANG */
    for (int q = 0; q < m; ++q) {
        int j = nb[q];
        double dj[3];
        displacement(xyz + 3 * i, xyz + 3 * j, cell, dj);
        double rj = sqrt(dot3(dj, dj));
        if (!(rj < RC_ANG)) continue;
        for (int w = q + 1; w < m; ++w) {
            int k = nb[w];
            double dk[3];
            displacement(xyz + 3 * i, xyz + 3 * k, cell, dk);
            double rk = sqrt(dot3(dk, dk));
            if (!(rk < RC_ANG)) continue;
            double cos_t = dot3(dj, dk) / (rj * rk);
            double theta = acos(0.95 * cos_t);
            double fcc = oracle_cutoff(rj, RC_ANG) * oracle_cutoff(rk, RC_ANG);
            int p = oracle_pair_index(species[j], species[k]);
            for (int a = 0; a < NASHIFT; ++a) {
                double t = 0.5 * (rj + rk) - angular_shift(a);
                double rad = exp(-ETA_ANG * t * t);
                for (int z = 0; z < NZSHIFT; ++z) {
                    double base = 0.5 * (1.0 + cos(theta - section_shift(z)));
                    G[RAD_LEN + 32 * p + 8 * a + z] += 2.0 * pow(base, ZETA) * rad * fcc;
                }
            }
        }
    }
}

/* AEVs of all atoms: G[n][1008]. */
void oracle_aev(int n, const int *species, const double *xyz, const double *cell, double *G)
{
    int *nb = (int *)malloc(sizeof(int) * (n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) aev_atom(i, n, species, xyz, cell, nb, G + (size_t)AEV_LEN * i);
    free(nb);
}

/* ------------------------------------------------------------ network */

/* Energy of one atom of element s from its AEV under net k of the ensemble;
 * if dEdG != NULL, also the gradient dE/dG (backpropagation through the four
 * layers). */
static double net_atom_energy(int s, const double *G, const oracle_weights *w, int k, double *dEdG)
{
    const size_t ks = (size_t)k * NSP + (size_t)s; /* (net, element) index */
    const double *W1 = w->W1 + ks * H1 * AEV_LEN, *b1 = w->b1 + ks * H1;
    const double *W2 = w->W2 + ks * H2 * H1, *b2 = w->b2 + ks * H2;
    const double *W3 = w->W3 + ks * H3 * H2, *b3 = w->b3 + ks * H3;
    const double *W4 = w->W4 + ks * H3, b4 = w->b4[ks];
    double z1[H1], h1[H1], z2[H2], h2[H2], z3[H3], h3[H3];
    for (int o = 0; o < H1; ++o) {
        double acc = b1[o];
        for (int c = 0; c < AEV_LEN; ++c) acc += W1[(size_t)o * AEV_LEN + c] * G[c];
        z1[o] = acc;
        h1[o] = oracle_celu(acc);
    }
    for (int o = 0; o < H2; ++o) {
        double acc = b2[o];
        for (int c = 0; c < H1; ++c) acc += W2[o * H1 + c] * h1[c];
        z2[o] = acc;
        h2[o] = oracle_celu(acc);
    }
    for (int o = 0; o < H3; ++o) {
        double acc = b3[o];
        for (int c = 0; c < H2; ++c) acc += W3[o * H2 + c] * h2[c];
        z3[o] = acc;
        h3[o] = oracle_celu(acc);
    }
    double e = b4;
    for (int c = 0; c < H3; ++c) e += W4[c] * h3[c];
    if (dEdG) {
        double g3[H3], g2[H2], g1[H1];
        for (int c = 0; c < H3; ++c) g3[c] = W4[c] * oracle_celu_deriv(z3[c]);
        for (int c = 0; c < H2; ++c) {
            double acc = 0.0;
            for (int o = 0; o < H3; ++o) acc += W3[o * H2 + c] * g3[o];
            g2[c] = acc * oracle_celu_deriv(z2[c]);
        }
        for (int c = 0; c < H1; ++c) {
            double acc = 0.0;
            for (int o = 0; o < H2; ++o) acc += W2[o * H1 + c] * g2[o];
            g1[c] = acc * oracle_celu_deriv(z1[c]);
        }
        for (int c = 0; c < AEV_LEN; ++c) {
            double acc = 0.0;
            for (int o = 0; o < H1; ++o) acc += W1[(size_t)o * AEV_LEN + c] * g1[o];
            dEdG[c] = acc;
        }
    }
    return e;
}

/* Energy of one atom of element s from its AEV, and optionally dE/dG. With an
 * ensemble of K independently trained nets the model is their average
 * (section "Performance of MLPs", the ANI-2x ensemble of eight, Table 3): e is
 * the mean of the K nets' energies and dE/dG the mean of their gradients, so
 * the forces are the mean of the K nets' forces. K = 1 is the single model. */
double oracle_atom_energy(int s, const double *G, const oracle_weights *w, double *dEdG)
{
    const int K = w->nets > 0 ? w->nets : 1;
    if (K == 1) return net_atom_energy(s, G, w, 0, dEdG);
    double gk[AEV_LEN];
    double e = 0.0;
    if (dEdG) memset(dEdG, 0, sizeof(double) * AEV_LEN);
    for (int k = 0; k < K; ++k) {
        e += net_atom_energy(s, G, w, k, dEdG ? gk : NULL);
        if (dEdG)
            for (int c = 0; c < AEV_LEN; ++c) dEdG[c] += gk[c];
    }
    if (dEdG)
        for (int c = 0; c < AEV_LEN; ++c) dEdG[c] /= K;
    return e / K;
}

/* ------------------------------------------------------------ forces */

/* Adds dE/dr contributions of atom i's AEV terms, given g = dE/dG_i, into
 * grad[n][3] (the gradient, i.e. minus the force). */
static void aev_atom_backward(int i, int n, const int *species, const double *xyz, const double *cell,
                              const double *g, int *nb, double *grad)
{
    int m = neighbors_of(i, n, xyz, cell, RC_RAD, nb);
    /* radial: dT/dr = 0.25 exp(-eta (r-R)^2) [-2 eta (r-R) fc + fc'] ; dr/dx_j = u, dr/dx_i = -u */
    for (int q = 0; q < m; ++q) {
        int j = nb[q];
        double d[3];
        displacement(xyz + 3 * i, xyz + 3 * j, cell, d);
        double r = sqrt(dot3(d, d));
        double fc = oracle_cutoff(r, RC_RAD), dfc = oracle_cutoff_deriv(r, RC_RAD);
        double s = 0.0;
        for (int k = 0; k < NRSHIFT; ++k) {
            double t = r - radial_shift(k);
            double gs = exp(-ETA_RAD * t * t);
            s += g[NRSHIFT * species[j] + k] * 0.25 * gs * (-2.0 * ETA_RAD * t * fc + dfc);
        }
        for (int c = 0; c < 3; ++c) {
            double v = s * d[c] / r;
            grad[3 * j + c] += v;
            grad[3 * i + c] -= v;
        }
    }
    /* angular */
    for (int q = 0; q < m; ++q) {
        int j = nb[q];
        double dj[3];
        displacement(xyz + 3 * i, xyz + 3 * j, cell, dj);
        double rj = sqrt(dot3(dj, dj));
        if (!(rj < RC_ANG)) continue;
        for (int w = q + 1; w < m; ++w) {
            int k = nb[w];
            double dk[3];
            displacement(xyz + 3 * i, xyz + 3 * k, cell, dk);
            double rk = sqrt(dot3(dk, dk));
            if (!(rk < RC_ANG)) continue;
            double djk = dot3(dj, dk);
            double c = 0.95 * djk / (rj * rk);
            double theta = acos(c);
            double dtheta_dc = -1.0 / sqrt(1.0 - c * c);
            double fj = oracle_cutoff(rj, RC_ANG), fk = oracle_cutoff(rk, RC_ANG);
            double dfj = oracle_cutoff_deriv(rj, RC_ANG), dfk = oracle_cutoff_deriv(rk, RC_ANG);
            int p = oracle_pair_index(species[j], species[k]);
            double S_c = 0.0, S_rj = 0.0, S_rk = 0.0;
            for (int a = 0; a < NASHIFT; ++a) {
                double t = 0.5 * (rj + rk) - angular_shift(a);
                double rad = exp(-ETA_ANG * t * t);
                double drad = -2.0 * ETA_ANG * t * rad * 0.5; /* d rad / d r_j = d rad / d r_k */
                for (int z = 0; z < NZSHIFT; ++z) {
                    double gg = g[RAD_LEN + 32 * p + 8 * a + z];
                    double base = 0.5 * (1.0 + cos(theta - section_shift(z)));
                    double P = 2.0 * pow(base, ZETA);
                    double dP_dtheta = 2.0 * ZETA * pow(base, ZETA - 1.0) * (-0.5 * sin(theta - section_shift(z)));
                    S_c += gg * dP_dtheta * dtheta_dc * rad * fj * fk;
                    S_rj += gg * P * (drad * fj * fk + rad * dfj * fk);
                    S_rk += gg * P * (drad * fj * fk + rad * fj * dfk);
                }
            }
            /* dc/d(dj) = 0.95 (dk / (rj rk) - (dj.dk) dj / (rj^3 rk)), symmetric for dk */
            for (int cc = 0; cc < 3; ++cc) {
                double dc_dj = 0.95 * (dk[cc] / (rj * rk) - djk * dj[cc] / (rj * rj * rj * rk));
                double dc_dk = 0.95 * (dj[cc] / (rj * rk) - djk * dk[cc] / (rk * rk * rk * rj));
                double gj = S_c * dc_dj + S_rj * dj[cc] / rj;
                double gk = S_c * dc_dk + S_rk * dk[cc] / rk;
                grad[3 * j + cc] += gj;
                grad[3 * k + cc] += gk;
                grad[3 * i + cc] -= gj + gk;
            }
        }
    }
}

/* Total energy; optional per-atom energies e_atoms[n]. */
double oracle_energy(int n, const int *species, const double *xyz, const double *cell,
                     const oracle_weights *w, double *e_atoms)
{
    double *G = (double *)malloc(sizeof(double) * AEV_LEN);
    int *nb = (int *)malloc(sizeof(int) * (n > 0 ? n : 1));
    double E = 0.0;
    for (int i = 0; i < n; ++i) {
        aev_atom(i, n, species, xyz, cell, nb, G);
        double e = oracle_atom_energy(species[i], G, w, NULL);
        if (e_atoms) e_atoms[i] = e;
        E += e;
    }
    free(G);
    free(nb);
    return E;
}

/* Total energy and forces F[n][3] = -dE/dr; optional per-atom energies. */
double oracle_energy_forces(int n, const int *species, const double *xyz, const double *cell,
                            const oracle_weights *w, double *e_atoms, double *F)
{
    double *G = (double *)malloc(sizeof(double) * AEV_LEN);
    double *g = (double *)malloc(sizeof(double) * AEV_LEN);
    int *nb = (int *)malloc(sizeof(int) * (n > 0 ? n : 1));
    double *grad = (double *)calloc((size_t)3 * (n > 0 ? n : 1), sizeof(double));
    double E = 0.0;
    for (int i = 0; i < n; ++i) {
        aev_atom(i, n, species, xyz, cell, nb, G);
        double e = oracle_atom_energy(species[i], G, w, g);
        if (e_atoms) e_atoms[i] = e;
        E += e;
        aev_atom_backward(i, n, species, xyz, cell, g, nb, grad);
    }
    for (int c = 0; c < 3 * n; ++c) F[c] = -grad[c];
    free(G);
    free(g);
    free(nb);
    free(grad);
    return E;
}

/* Forces F[n][3] = -sum_i dEdG_i . dG_i/dr for a given dE/dG (dEdG[n][1008],
 * row i belonging to atom i): the AEV backward alone, the chain rule below
 * the network (section "PyTorch Model Support": forces by backpropagation).
 * With dE/dG from the oracle's own network it equals the forces of
 * oracle_energy_forces. */
void oracle_forces_from_dEdG(int n, const int *species, const double *xyz, const double *cell,
                             const double *dEdG, double *F)
{
    int *nb = (int *)malloc(sizeof(int) * (n > 0 ? n : 1));
    double *grad = (double *)calloc((size_t)3 * (n > 0 ? n : 1), sizeof(double));
    for (int i = 0; i < n; ++i)
        aev_atom_backward(i, n, species, xyz, cell, dEdG + (size_t)AEV_LEN * i, nb, grad);
    for (int c = 0; c < 3 * n; ++c) F[c] = -grad[c];
    free(nb);
    free(grad);
}

/* dE/dG for every atom: dEdG[n][1008], and e_atoms[n]. */
void oracle_aev_grad(int n, const int *species, const double *xyz, const double *cell,
                     const oracle_weights *w, double *e_atoms, double *dEdG)
{
    double *G = (double *)malloc(sizeof(double) * AEV_LEN);
    int *nb = (int *)malloc(sizeof(int) * (n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) {
        aev_atom(i, n, species, xyz, cell, nb, G);
        double e = oracle_atom_energy(species[i], G, w, dEdG + (size_t)AEV_LEN * i);
        if (e_atoms) e_atoms[i] = e;
    }
    free(G);
    free(nb);
}

/* Forces on a subset of atoms, F_sub[nsub][3]. The AEV of atom i depends on
 * the position of atom m only when i == m or |d_im| < Rc_R, so only those
 * atoms' terms are evaluated; the result equals the matching rows of
 * oracle_energy_forces. */
void oracle_forces_subset(int n, const int *species, const double *xyz, const double *cell,
                          const oracle_weights *w, int nsub, const int *idx, double *F_sub)
{
    double *G = (double *)malloc(sizeof(double) * AEV_LEN);
    double *g = (double *)malloc(sizeof(double) * AEV_LEN);
    int *nb = (int *)malloc(sizeof(int) * (n > 0 ? n : 1));
    int *around = (int *)malloc(sizeof(int) * (n > 0 ? n : 1));
    double *grad = (double *)calloc((size_t)3 * (n > 0 ? n : 1), sizeof(double));
    for (int s = 0; s < nsub; ++s) {
        int m = idx[s];
        int cnt = neighbors_of(m, n, xyz, cell, RC_RAD, around);
        around[cnt++] = m;
        memset(grad, 0, sizeof(double) * 3 * (size_t)n);
        for (int q = 0; q < cnt; ++q) {
            int i = around[q];
            aev_atom(i, n, species, xyz, cell, nb, G);
            oracle_atom_energy(species[i], G, w, g);
            aev_atom_backward(i, n, species, xyz, cell, g, nb, grad);
        }
        for (int c = 0; c < 3; ++c) F_sub[3 * s + c] = -grad[3 * m + c];
    }
    free(G);
    free(g);
    free(nb);
    free(around);
    free(grad);
}

/* Sum of e_i over atom m and every atom within Rc_R + margin of it: the part
 * of E that moves when atom m moves by less than margin (for finite
 * differences on large systems). */
double oracle_local_energy(int n, const int *species, const double *xyz, const double *cell,
                           const oracle_weights *w, int m, const double *center, double margin)
{
    double *G = (double *)malloc(sizeof(double) * AEV_LEN);
    int *nb = (int *)malloc(sizeof(int) * (n > 0 ? n : 1));
    double E = 0.0;
    double lim = RC_RAD + margin;
    for (int i = 0; i < n; ++i) {
        double d[3];
        displacement(center, xyz + 3 * i, cell, d);
        if (i != m && !(dot3(d, d) < lim * lim)) continue;
        aev_atom(i, n, species, xyz, cell, nb, G);
        E += oracle_atom_energy(species[i], G, w, NULL);
    }
    free(G);
    free(nb);
    return E;
}

/* ML/MM mechanical embedding (section "OpenMM-ML": a listed subset of the
 * atoms is modeled by the MLP; the rest, and the interaction between the two
 * regions, by a conventional force field). The ML part of the energy is the
 * potential of the subset alone: E_ML = E(species[index], xyz[index]) with the
 * system's cell; its forces act on the subset only. F_full[n_full][3] receives
 * them in rows index[q] and zeros everywhere else. */
double oracle_ml_region(int n_full, const int *species, const double *xyz, const double *cell,
                        const oracle_weights *w, int n_ml, const int *index, double *F_full)
{
    int *sp = (int *)malloc(sizeof(int) * (n_ml > 0 ? n_ml : 1));
    double *x = (double *)malloc(sizeof(double) * 3 * (n_ml > 0 ? n_ml : 1));
    double *F = (double *)malloc(sizeof(double) * 3 * (n_ml > 0 ? n_ml : 1));
    for (int q = 0; q < n_ml; ++q) {
        sp[q] = species[index[q]];
        for (int c = 0; c < 3; ++c) x[3 * q + c] = xyz[3 * index[q] + c];
    }
    double E = oracle_energy_forces(n_ml, sp, x, cell, w, NULL, F);
    for (int c = 0; c < 3 * n_full; ++c) F_full[c] = 0.0;
    for (int q = 0; q < n_ml; ++q)
        for (int c = 0; c < 3; ++c) F_full[3 * index[q] + c] = F[3 * q + c];
    free(sp);
    free(x);
    free(F);
    return E;
}

/* Independent molecules back to back (atoms mol_start[m] .. mol_start[m+1]),
 * each evaluated by oracle_energy_forces; cells[3 m] per molecule or NULL.
 * Molecules are spread over nthreads OpenMP threads when built with OpenMP. */
void oracle_energy_forces_batch(int nmol, const long *mol_start, const int *species, const double *xyz,
                                const double *cells, const oracle_weights *w, double *E, double *F,
                                int nthreads)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int m = 0; m < nmol; ++m) {
        long a = mol_start[m], b = mol_start[m + 1];
        E[m] = oracle_energy_forces((int)(b - a), species + a, xyz + 3 * a, cells ? cells + 3 * m : NULL, w,
                                    NULL, F + 3 * a);
    }
    (void)nthreads;
}

/* Per-atom energies e_out[q] = e_{idx[q]} for the listed atoms (each one an
 * independent evaluation of its AEV and network), spread over nthreads
 * OpenMP threads when built with OpenMP. */
void oracle_atom_energies(int n, const int *species, const double *xyz, const double *cell,
                          const oracle_weights *w, int nidx, const int *idx, double *e_out, int nthreads)
{
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1)
#endif
    {
        double *G = (double *)malloc(sizeof(double) * AEV_LEN);
        int *nb = (int *)malloc(sizeof(int) * (n > 0 ? n : 1));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
        for (int q = 0; q < nidx; ++q) {
            int i = idx[q];
            aev_atom(i, n, species, xyz, cell, nb, G);
            e_out[q] = oracle_atom_energy(species[i], G, w, NULL);
        }
        free(G);
        free(nb);
    }
    (void)nthreads;
}

/* AEV rows of the listed atoms only: G_out[nidx][1008]. */
void oracle_aev_subset(int n, const int *species, const double *xyz, const double *cell, int nidx, const int *idx,
                       double *G_out)
{
    int *nb = (int *)malloc(sizeof(int) * (n > 0 ? n : 1));
    for (int q = 0; q < nidx; ++q) aev_atom(idx[q], n, species, xyz, cell, nb, G_out + (size_t)AEV_LEN * q);
    free(nb);
}

/* ------------------------------------------------------------ Langevin dynamics */
/* Section "New Integrators": the LF-Middle discretization of the Langevin
 * equation; section "Performance of MLPs" (Table 3): the ML simulations run
 * with a Langevin integrator and a 2 fs step. One step, velocities at half
 * steps (leapfrog), forces F(x_t):
 *   v <- v + dt F / m                      (v: t - dt/2 -> t + dt/2)
 *   x <- x + (dt / 2) v
 *   v <- a v + sqrt((1 - a^2) kT / m) R,   a = exp(-gamma dt), R ~ N(0, 1)
 *   x <- x + (dt / 2) v
 * Units: A, fs, amu, eV; F / m in eV / (A amu) = 9.648533212e-3 A / fs^2;
 * kT / m in eV / amu = 1 / 103.6426965 A^2 / fs^2.
 * The normal deviates are drawn from Philox4x64-10 (Salmon, Moraes, Dror,
 * Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC 2011): atom i at
 * step t uses counter (t, i, 0, 0) and key (seed, 0); its four 64-bit words
 * give uniforms u = (w >> 11) 2^-53 and, by Box-Muller on the pairs (0, 1)
 * and (2, 3), normals R_x, R_y, R_z (the fourth is unused):
 *   r = sqrt(-2 ln(1 - u_a)), R = r cos(2 pi u_b), r sin(2 pi u_b). */

static const double LGV_ACC = 9.648533212e-3;
static const double LGV_KE = 103.6426965;
static const double LGV_KB = 8.617333262e-5;
static const double LGV_MASS[NSP] = {1.008, 12.011, 14.007, 15.999, 32.06, 18.998, 35.45};

static void mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo)
{
    unsigned __int128 p = (unsigned __int128)a * b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

/* Philox4x64 with 10 rounds (the published definition). */
void oracle_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3], k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(0xD2E7470EE14C6C93ull, c0, &hi0, &lo0);
        mulhilo64(0xCA5A826395121157ull, c2, &hi1, &lo1);
        const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B97F4A7C15ull; /* Weyl sequence: golden ratio */
        k1 += 0xBB67AE8584CAA73Bull; /* sqrt(3) - 1 */
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* The three normal deviates of atom i at step t (see above). */
void oracle_langevin_normals(uint64_t seed, int64_t step, int atom, double R[3])
{
    const uint64_t ctr[4] = {(uint64_t)step, (uint64_t)atom, 0, 0}, key[2] = {seed, 0};
    uint64_t w[4];
    oracle_philox4x64(ctr, key, w);
    double u[4];
    for (int q = 0; q < 4; ++q) u[q] = (double)(w[q] >> 11) * 0x1.0p-53;
    const double r0 = sqrt(-2.0 * log(1.0 - u[0])), r1 = sqrt(-2.0 * log(1.0 - u[2]));
    R[0] = r0 * cos(2.0 * M_PI * u[1]);
    R[1] = r0 * sin(2.0 * M_PI * u[1]);
    R[2] = r1 * cos(2.0 * M_PI * u[3]);
}

/* One LF-Middle update of n atoms from forces F (eV / A); dt in fs, gamma in
 * 1 / ps, temperature in K. x and v are updated in place. */
void oracle_lfmiddle_step(int n, const int *species, double *x, double *v, const double *F, double dt,
                          double gamma_per_ps, double temperature, uint64_t seed, int64_t step)
{
    const double a = exp(-gamma_per_ps * 1e-3 * dt);
    const double kT = LGV_KB * temperature;
    for (int i = 0; i < n; ++i) {
        const double m = LGV_MASS[species[i]];
        const double sig = sqrt((1.0 - a * a) * kT / (m * LGV_KE));
        double R[3];
        oracle_langevin_normals(seed, step, i, R);
        for (int c = 0; c < 3; ++c) {
            double vv = v[3 * i + c] + dt * F[3 * i + c] * LGV_ACC / m;
            double xx = x[3 * i + c] + 0.5 * dt * vv;
            vv = a * vv + sig * R[c];
            xx += 0.5 * dt * vv;
            v[3 * i + c] = vv;
            x[3 * i + c] = xx;
        }
    }
}

/* n_steps LF-Middle steps with the oracle's forces, starting at step index
 * step0; E_pot[s] = potential energy at the start of step s (may be NULL). */
void oracle_langevin_run(int n, const int *species, double *x, double *v, const double *cell,
                         const oracle_weights *w, double dt, double gamma_per_ps, double temperature,
                         uint64_t seed, int64_t step0, int n_steps, double *E_pot)
{
    double *F = (double *)malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
    for (int s = 0; s < n_steps; ++s) {
        const double E = oracle_energy_forces(n, species, x, cell, w, NULL, F);
        if (E_pot) E_pot[s] = E;
        oracle_lfmiddle_step(n, species, x, v, F, dt, gamma_per_ps, temperature, seed, step0 + s);
    }
    free(F);
}

int oracle_aev_length(void) { return AEV_LEN; }
