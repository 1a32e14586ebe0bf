/*
 * Seeded synthetic workload generator: ligand trees and pocket grids.
 *
 * This file builds INPUTS only.  It holds none of the docking arithmetic
 * (no pose sampling, no torsion sweep, no interpolation, no scoring): both the
 * FP64 oracle and the CUDA path consume what it writes, and neither links it.
 *
 * The paper describes its inputs only qualitatively: ligands of tens of atoms
 * and up to tens of torsional bonds (Sec. 3.1), a rigid binding site whose
 * description is read once (Sec. 3.2), 3D ligand structures with positions,
 * types and bonds (Sec. 4.1).  The concrete recipe below (tree growth, bond
 * lengths and angles, clash rejection, type mix, grid potentials) is this
 * project's synthetic stand-in for the paper's chemical library and PDB pockets.
 *
 * Randomness: xoshiro256** (Blackman & Vigna, 2018) seeded through splitmix64,
 * one independent stream per ligand, so results do not depend on thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ---------------- PRNG ---------------- */
typedef struct { uint64_t s[4]; } xs_t;

static uint64_t splitmix64(uint64_t *x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static void xs_seed(xs_t *r, uint64_t seed) {
    uint64_t x = seed;
    for (int i = 0; i < 4; i++) r->s[i] = splitmix64(&x);
}
static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }
static uint64_t xs_next(xs_t *r) {
    uint64_t *s = r->s;
    uint64_t res = rotl64(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3];
    s[2] ^= t; s[3] = rotl64(s[3], 45);
    return res;
}
static double xs_u01(xs_t *r) { return (double)(xs_next(r) >> 11) * 0x1.0p-53; }
static int xs_below(xs_t *r, int n) {
    int v = (int)(xs_u01(r) * n);
    return v < n ? v : n - 1;
}
static double xs_normal(xs_t *r) {
    double u1 = xs_u01(r), u2 = xs_u01(r);
    if (u1 < 1e-300) u1 = 1e-300;
    return sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
}
static void xs_unit(xs_t *r, double v[3]) {
    for (;;) {
        v[0] = xs_normal(r); v[1] = xs_normal(r); v[2] = xs_normal(r);
        double n2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
        if (n2 > 1e-12) {
            double inv = 1.0 / sqrt(n2);
            v[0] *= inv; v[1] *= inv; v[2] *= inv;
            return;
        }
    }
}

/* ---------------- ligand trees ---------------- */
#define SY_MAXN 256

/* Growth recipe (per atom i >= 1):
 *   parent p uniform among placed atoms with fewer than 4 bonds;
 *   bond length U(1.45, 1.55) A;
 *   if p already has a neighbour nb: angle(nb-p-i) ~ U(104.5, 114.5) deg with a
 *   uniform dihedral about p->nb; else a uniform direction;
 *   the placement is rejected when the new atom lies closer than `min_sep` to
 *   any placed atom other than p (this covers 1-3 pairs with an uncontrolled
 *   angle and every pair three or more bonds apart); 100 tries, then the whole
 *   ligand is redrawn.
 * Atoms are then renumbered in depth-first preorder from atom 0 (children in
 * creation order), so parent[i] < i and every subtree is a contiguous range. */
static int grow_tree(xs_t *r, int N, double min_sep, double pos[][3], int par[]) {
    int deg[SY_MAXN];
    int nbr[SY_MAXN][4];
    for (int attempt = 0; attempt < 1000; attempt++) {
        memset(deg, 0, sizeof(int) * N);
        pos[0][0] = pos[0][1] = pos[0][2] = 0.0;
        par[0] = -1;
        int ok_all = 1;
        for (int i = 1; i < N && ok_all; i++) {
            int placed = 0;
            for (int tries = 0; tries < 100 && !placed; tries++) {
                int cand[SY_MAXN], nc = 0;
                for (int j = 0; j < i; j++)
                    if (deg[j] < 4) cand[nc++] = j;
                if (nc == 0) break;
                int p = cand[xs_below(r, nc)];
                double L = 1.45 + 0.10 * xs_u01(r);
                double d[3];
                if (deg[p] == 0) {
                    xs_unit(r, d);
                } else {
                    int nb = nbr[p][xs_below(r, deg[p])];
                    double rv[3] = {pos[nb][0] - pos[p][0], pos[nb][1] - pos[p][1], pos[nb][2] - pos[p][2]};
                    double rn = sqrt(rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2]);
                    rv[0] /= rn; rv[1] /= rn; rv[2] /= rn;
                    /* orthonormal n1, n2 perpendicular to rv */
                    double t[3];
                    xs_unit(r, t);
                    double dt = t[0] * rv[0] + t[1] * rv[1] + t[2] * rv[2];
                    double n1[3] = {t[0] - dt * rv[0], t[1] - dt * rv[1], t[2] - dt * rv[2]};
                    double n1n = sqrt(n1[0] * n1[0] + n1[1] * n1[1] + n1[2] * n1[2]);
                    if (n1n < 1e-6) continue;
                    n1[0] /= n1n; n1[1] /= n1n; n1[2] /= n1n;
                    double n2[3] = {rv[1] * n1[2] - rv[2] * n1[1], rv[2] * n1[0] - rv[0] * n1[2],
                                    rv[0] * n1[1] - rv[1] * n1[0]};
                    double alpha = (104.5 + 10.0 * xs_u01(r)) * M_PI / 180.0;
                    double phi = 2.0 * M_PI * xs_u01(r);
                    double ca = cos(alpha), sa = sin(alpha), cp = cos(phi), sp = sin(phi);
                    for (int c = 0; c < 3; c++) d[c] = rv[c] * ca + (n1[c] * cp + n2[c] * sp) * sa;
                }
                double x[3] = {pos[p][0] + L * d[0], pos[p][1] + L * d[1], pos[p][2] + L * d[2]};
                int ok = 1;
                for (int j = 0; j < i && ok; j++) {
                    if (j == p) continue;
                    double dx = x[0] - pos[j][0], dy = x[1] - pos[j][1], dz = x[2] - pos[j][2];
                    if (dx * dx + dy * dy + dz * dz < min_sep * min_sep) ok = 0;
                }
                if (!ok) continue;
                pos[i][0] = x[0]; pos[i][1] = x[1]; pos[i][2] = x[2];
                par[i] = p;
                nbr[p][deg[p]++] = i;
                nbr[i][deg[i]++] = p;
                placed = 1;
            }
            if (!placed) ok_all = 0;
        }
        if (ok_all) return 0;
    }
    return -1;
}

/* Depth-first preorder renumbering (children visited in creation order). */
static void preorder(int N, double pos[][3], int par[], double out_pos[][3], int out_par[]) {
    int first_child[SY_MAXN], next_sib[SY_MAXN], last_child[SY_MAXN];
    for (int i = 0; i < N; i++) first_child[i] = next_sib[i] = last_child[i] = -1;
    for (int i = 1; i < N; i++) {
        int p = par[i];
        if (first_child[p] < 0) first_child[p] = i; else next_sib[last_child[p]] = i;
        last_child[p] = i;
    }
    int newid[SY_MAXN], stack[SY_MAXN], sp = 0, next = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        int v = stack[--sp];
        newid[v] = next++;
        /* push children in reverse creation order so the first child is visited first */
        int ch[SY_MAXN], nch = 0;
        for (int c = first_child[v]; c >= 0; c = next_sib[c]) ch[nch++] = c;
        for (int k = nch - 1; k >= 0; k--) stack[sp++] = ch[k];
    }
    for (int i = 0; i < N; i++) {
        int ni = newid[i];
        out_pos[ni][0] = pos[i][0]; out_pos[ni][1] = pos[i][1]; out_pos[ni][2] = pos[i][2];
        out_par[ni] = (par[i] < 0) ? -1 : newid[par[i]];
    }
}

/* One ligand.  Writes N atoms and up to N rotatable-bond children (ascending).
 * Rotatable bonds: tree bonds (parent(b), b) whose two atoms both have >= 2
 * bonds; a uniform random subset of min(R_target, eligible) of them is kept.
 * Types C/N/O/S/Cl = 0..4 at 70/12/12/3/3 %; charges N(0, 0.2) minus their mean.
 * The whole ligand is translated by U(-offset, offset) per axis.
 * Returns the number of rotatable bonds written, or -1 on failure. */
int synth_ligand(uint64_t seed, int N, int R_target, double offset, double min_sep,
                 float *x, float *y, float *z, float *q, uint8_t *type, int16_t *parent,
                 int16_t *rot_child) {
    if (N < 1 || N > SY_MAXN) return -1;
    xs_t r;
    xs_seed(&r, seed);
    static __thread double pos[SY_MAXN][3], pos2[SY_MAXN][3];
    int par[SY_MAXN], par2[SY_MAXN];
    if (grow_tree(&r, N, min_sep, pos, par) != 0) return -1;
    preorder(N, pos, par, pos2, par2);
    double off[3];
    for (int c = 0; c < 3; c++) off[c] = offset * (2.0 * xs_u01(&r) - 1.0);
    double qsum = 0.0, qq[SY_MAXN];
    for (int i = 0; i < N; i++) {
        x[i] = (float)(pos2[i][0] + off[0]);
        y[i] = (float)(pos2[i][1] + off[1]);
        z[i] = (float)(pos2[i][2] + off[2]);
        parent[i] = (int16_t)par2[i];
        double u = xs_u01(&r);
        type[i] = (uint8_t)(u < 0.70 ? 0 : u < 0.82 ? 1 : u < 0.94 ? 2 : u < 0.97 ? 3 : 4);
        qq[i] = 0.2 * xs_normal(&r);
        qsum += qq[i];
    }
    for (int i = 0; i < N; i++) q[i] = (float)(qq[i] - qsum / N);
    int deg[SY_MAXN];
    memset(deg, 0, sizeof(int) * N);
    for (int i = 1; i < N; i++) { deg[i]++; deg[par2[i]]++; }
    int elig[SY_MAXN], ne = 0;
    for (int b = 1; b < N; b++)
        if (deg[b] >= 2 && deg[par2[b]] >= 2) elig[ne++] = b;
    int R = R_target < ne ? R_target : ne;
    if (R < 0) R = 0;
    for (int k = 0; k < R; k++) { /* partial Fisher-Yates */
        int j = k + xs_below(&r, ne - k);
        int t = elig[k]; elig[k] = elig[j]; elig[j] = t;
    }
    /* sort the chosen R ascending (insertion sort, R is small) */
    for (int k = 1; k < R; k++) {
        int v = elig[k], j = k - 1;
        while (j >= 0 && elig[j] > v) { elig[j + 1] = elig[j]; j--; }
        elig[j + 1] = v;
    }
    for (int k = 0; k < R; k++) rot_child[k] = (int16_t)elig[k];
    return R;
}

/* Batch of ligands in CSR layout.  rot_tmp has one slot per atom (atom_off
 * indexing); R_out[l] tells how many of ligand l's slots are used. */
int synth_ligands(int L, const uint64_t *seeds, const int32_t *Rt, const int32_t *atom_off,
                  double offset, double min_sep, float *x, float *y, float *z, float *q,
                  uint8_t *type, int16_t *parent, int16_t *rot_tmp, int32_t *R_out) {
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : bad)
    for (int l = 0; l < L; l++) {
        int a0 = atom_off[l], N = atom_off[l + 1] - a0;
        int R = synth_ligand(seeds[l], N, Rt[l], offset, min_sep, x + a0, y + a0, z + a0, q + a0,
                             type + a0, parent + a0, rot_tmp + a0);
        R_out[l] = R;
        if (R < 0) bad++;
    }
    return bad;
}

/* ---------------- pocket grids ---------------- */

/* Pocket points: grid nodes strictly inside the cavity ellipsoid (about
 * cav_center, semi-axes cav_radii) that are at least `clear` A from every
 * protein atom.  Writes node indices (i, j, k) and returns their count. */
int synth_pocket_points(int n, double h, const double *origin, int na, const double *axyz,
                        const double *cav_center, const double *cav_radii, double clear,
                        int32_t *pp_out) {
    int npp = 0;
    for (int k = 0; k < n; k++)
        for (int j = 0; j < n; j++)
            for (int i = 0; i < n; i++) {
                double g[3] = {origin[0] + h * i, origin[1] + h * j, origin[2] + h * k};
                double rho = 0.0;
                for (int c = 0; c < 3; c++) {
                    double t = (g[c] - cav_center[c]) / cav_radii[c];
                    rho += t * t;
                }
                if (rho >= 1.0) continue;
                int ok = 1;
                for (int a = 0; a < na && ok; a++) {
                    double dx = g[0] - axyz[3 * a], dy = g[1] - axyz[3 * a + 1], dz = g[2] - axyz[3 * a + 2];
                    if (dx * dx + dy * dy + dz * dz < clear * clear) ok = 0;
                }
                if (!ok) continue;
                pp_out[3 * npp] = i; pp_out[3 * npp + 1] = j; pp_out[3 * npp + 2] = k;
                npp++;
            }
    return npp;
}

/* Pocket-overlap field: sum over pocket points of exp(-d^2 / (2 sigma^2)) for
 * d <= cut, then divided by its maximum so it lies in [0, 1]. */
void synth_overlap_grid(int n, double h, int npp, const int32_t *pp, double sigma, double cut,
                        double *phi) {
    size_t n3 = (size_t)n * n * n;
    for (size_t t = 0; t < n3; t++) phi[t] = 0.0;
    int w = (int)ceil(cut / h);
    for (int p = 0; p < npp; p++) {
        int pi = pp[3 * p], pj = pp[3 * p + 1], pk = pp[3 * p + 2];
        for (int k = pk - w; k <= pk + w; k++) {
            if (k < 0 || k >= n) continue;
            for (int j = pj - w; j <= pj + w; j++) {
                if (j < 0 || j >= n) continue;
                for (int i = pi - w; i <= pi + w; i++) {
                    if (i < 0 || i >= n) continue;
                    double dx = h * (i - pi), dy = h * (j - pj), dz = h * (k - pk);
                    double d2 = dx * dx + dy * dy + dz * dz;
                    if (d2 > cut * cut) continue;
                    phi[((size_t)k * n + j) * n + i] += exp(-d2 / (2.0 * sigma * sigma));
                }
            }
        }
    }
    double mx = 0.0;
    for (size_t t = 0; t < n3; t++) if (phi[t] > mx) mx = phi[t];
    if (mx > 0.0)
        for (size_t t = 0; t < n3; t++) phi[t] /= mx;
}

/* Direct pairwise potentials of a set of protein atoms at one point.
 *   vdw  = min(cap, sum_{r < cut_v} eps * ((r0/r)^12 - 2 (r0/r)^6)),  r >= rmin_v
 *   elec = sum_{r < cut_e} kel * q_j / (4 r^2),                       r >= rmin_e
 * (Lennard-Jones well of depth eps at r0; distance-dependent dielectric 4r.) */
typedef struct {
    double eps, r0, cut_v, cap_v, rmin_v, kel, cut_e, rmin_e;
} sy_pot;

static void point_potentials(const double g[3], int na, const double *axyz, const double *aq,
                             const sy_pot *P, double *vdw, double *elec) {
    double v = 0.0, e = 0.0;
    for (int a = 0; a < na; a++) {
        double dx = g[0] - axyz[3 * a], dy = g[1] - axyz[3 * a + 1], dz = g[2] - axyz[3 * a + 2];
        double d2 = dx * dx + dy * dy + dz * dz;
        if (d2 < P->cut_v * P->cut_v) {
            double r = sqrt(d2);
            if (r < P->rmin_v) r = P->rmin_v;
            double s = P->r0 / r, s2 = s * s, s6 = s2 * s2 * s2;
            v += P->eps * (s6 * s6 - 2.0 * s6);
        }
        if (d2 < P->cut_e * P->cut_e) {
            double r2 = d2 < P->rmin_e * P->rmin_e ? P->rmin_e * P->rmin_e : d2;
            e += P->kel * aq[a] / (4.0 * r2);
        }
    }
    *vdw = v < P->cap_v ? v : P->cap_v;
    *elec = e;
}

/* Potentials at arbitrary points (npts x 3, A). */
void synth_direct_potentials(int npts, const double *pts, int na, const double *axyz, const double *aq,
                             double eps, double r0, double cut_v, double cap_v, double rmin_v,
                             double kel, double cut_e, double rmin_e, double *vdw, double *elec) {
    sy_pot P = {eps, r0, cut_v, cap_v, rmin_v, kel, cut_e, rmin_e};
#pragma omp parallel for schedule(static)
    for (int p = 0; p < npts; p++) point_potentials(pts + 3 * p, na, axyz, aq, &P, vdw + p, elec + p);
}

/* Potentials at every grid node (x fastest): node (i,j,k) sits at origin + h*(i,j,k). */
void synth_potential_grids(int n, double h, const double *origin, int na, const double *axyz,
                           const double *aq, double eps, double r0, double cut_v, double cap_v,
                           double rmin_v, double kel, double cut_e, double rmin_e, double *phi_v,
                           double *phi_e) {
    sy_pot P = {eps, r0, cut_v, cap_v, rmin_v, kel, cut_e, rmin_e};
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < n; k++)
        for (int j = 0; j < n; j++)
            for (int i = 0; i < n; i++) {
                double g[3] = {origin[0] + h * i, origin[1] + h * j, origin[2] + h * k};
                size_t t = ((size_t)k * n + j) * n + i;
                point_potentials(g, na, axyz, aq, &P, phi_v + t, phi_e + t);
            }
}
