/*
 * FP64 CPU oracle of the dock-and-score hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg load it; the library never does.  It shares no
 * code, header, table or constant with the CUDA path.
 *
 * What it computes (the paper's dock-and-score step, Sec. 3.1): a ligand is
 * docked in a rigid pocket by a greedy optimisation with multiple restarts
 * driven by a purely geometric (steric) score; the ligand is flexible through
 * its torsional bonds, each of which splits the atoms into two sets that can
 * turn about the bond axis; torsional bonds are processed one after the other
 * (Sec. 3.1, the GPU discussion); the ligand's score is the score of its best
 * pose.  The paper gives no formulas, so the concrete steps are readings,
 * applied identically on both sides:
 *
 *   pose    For restart r of ligand uid: Philox4x32-10 (Salmon et al., SC'11)
 *           with key (seed_lo, seed_hi) and counter (uid_lo, uid_hi, r, 0) gives
 *           four words x0..x3; u_i = (x_i >> 8) * 2^-24; Shoemake's uniform
 *           quaternion from (u0, u1, u2) gives R; the pocket point index is
 *           ((x3 >> 8) * n_pp) >> 24; atoms go to R (x - c) + p with c the
 *           unweighted centroid and p the pocket point's node position.
 *   sweep   For pass = 0..P-1 and torsional bond k in ascending child order:
 *           the bond (a = parent(b), b); moving set M = subtree(b) minus b,
 *           fixed set F = atoms outside subtree(b).  For angle step t = 0..A-1
 *           (theta = 2 pi t / A) the moving atoms turn about the axis a->b
 *           through b (right-hand rule); the overlap score is the sum over M of
 *           the trilinearly interpolated overlap grid.  Step t is admissible
 *           when t = 0 (the current pose) or every pair (i in M, j in F) that is
 *           at least three bonds apart is at least d_clash apart.  The chosen
 *           step is the admissible one with the largest score, the lowest step
 *           on ties; it is applied when it is not 0.
 *   rigid   (optional) After each torsion pass, rigid_steps greedy rigid moves of
 *           the whole ligand: candidate 0 stays; 1..6 translate by +d, -d along
 *           x, y, z (d = rigid_shift); 7..12 turn by +a, -a (a = 2 pi / A) about
 *           the x, y, z axes through the ligand's centroid (right-hand rule).
 *           The candidate with the largest geometric score G = sum over all
 *           atoms of the overlap grid wins, the lowest candidate on ties.
 *   score   E = sum_i [ w_type(i) Vgrid(xhat_i) + q_i Egrid(xhat_i) + k_out |x_i - xhat_i| ]
 *           with xhat the position clamped to the grid box.
 *   best    The restart with the lowest E wins, the lowest restart on ties.
 *   flatten (separate entry, Sec. 3.1 step 1) The same greedy sweep, without
 *           a pocket, maximising the sum of all pairwise atom distances.
 *   rank    (optional, Sec. 3.1 steps 3-4) The poses are ordered by geometric
 *           score G = sum over all atoms of the overlap grid (higher first,
 *           lower restart on ties) and clustered greedily: a pose whose RMSD
 *           (no superposition) to an earlier cluster leader is at most the
 *           threshold joins the first such leader, otherwise it leads a new
 *           cluster.  The ranking lists the leaders in order, then the other
 *           poses in order; the first K ranked poses are rescored and the one
 *           with the lowest E (lowest restart on ties) is the ligand's result.
 *
 * Trilinear interpolation (textbook definition): node (i,j,k) at origin +
 * h (i,j,k), flat index (k n + j) n + i; g = (xhat - origin)/h; i0 =
 * min(floor(g), n-2); f = g - i0; lerp along x, then y, then z.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define OR_MAXN 256

typedef struct {
    int32_t n;
    double h;
    double origin[3];
    const float *phi_o, *phi_v, *phi_e; /* n^3 each, x fastest */
    int32_t n_pp;
    const int32_t *pp; /* [n_pp][3] node indices */
    double type_w[5];
    double k_out;
} or_pocket;

typedef struct {
    int32_t restarts, passes, angle_steps;
    uint64_t seed;
    double d_clash;
    double cluster_rmsd; /* 0: no clustering */
    int32_t rescore_top; /* K; 0 or >= restarts: all poses */
    int32_t rigid_steps; /* rigid greedy moves after each torsion pass (0: none) */
    double rigid_shift;  /* translation step of a rigid move (A) */
} or_params;

/* ------------------------------------------------------------------ Philox4x32-10
 * Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
 * SC'11: ten rounds of the Philox S-box on a 4 x 32-bit counter with a 2 x 32-bit
 * key; each round multiplies words 0 and 2 by the two round constants, keeps
 * both product halves, mixes the high halves with the other two words and the
 * key, and the key is bumped by the two Weyl constants between rounds. */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        uint64_t p0 = (uint64_t)M0 * c0;
        uint64_t p1 = (uint64_t)M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0; k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* A 24-bit uniform in [0, 1), exact in both FP32 and FP64. */
static double u24(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }

/* ------------------------------------------------------------------ Shoemake rotation
 * K. Shoemake, "Uniform random rotations", Graphics Gems III (1992): with
 * s1 = sqrt(1-u0), s2 = sqrt(u0), the quaternion (x, y, z, w) =
 * (s1 sin 2pi u1, s1 cos 2pi u1, s2 sin 2pi u2, s2 cos 2pi u2) is uniform on the
 * unit 3-sphere; R is the rotation matrix of the unit quaternion w + xi + yj + zk
 * (row-major). */
void or_shoemake(double u0, double u1, double u2, double R[9]) {
    double s1 = sqrt(1.0 - u0), s2 = sqrt(u0);
    double qx = s1 * sin(2.0 * M_PI * u1), qy = s1 * cos(2.0 * M_PI * u1);
    double qz = s2 * sin(2.0 * M_PI * u2), qw = s2 * cos(2.0 * M_PI * u2);
    R[0] = 1.0 - 2.0 * (qy * qy + qz * qz);
    R[1] = 2.0 * (qx * qy - qw * qz);
    R[2] = 2.0 * (qx * qz + qw * qy);
    R[3] = 2.0 * (qx * qy + qw * qz);
    R[4] = 1.0 - 2.0 * (qx * qx + qz * qz);
    R[5] = 2.0 * (qy * qz - qw * qx);
    R[6] = 2.0 * (qx * qz - qw * qy);
    R[7] = 2.0 * (qy * qz + qw * qx);
    R[8] = 1.0 - 2.0 * (qx * qx + qy * qy);
}

/* Rotation and pocket point of restart r (the "pose" reading above). */
void or_restart_pose(const or_pocket *P, const or_params *prm, uint64_t uid, int32_t r, double R[9],
                     double p[3], int32_t *pp_index) {
    uint32_t ctr[4] = {(uint32_t)uid, (uint32_t)(uid >> 32), (uint32_t)r, 0u};
    uint32_t key[2] = {(uint32_t)prm->seed, (uint32_t)(prm->seed >> 32)};
    uint32_t x[4];
    or_philox4x32_10(ctr, key, x);
    or_shoemake(u24(x[0]), u24(x[1]), u24(x[2]), R);
    int32_t idx = (int32_t)(((uint64_t)(x[3] >> 8) * (uint64_t)P->n_pp) >> 24);
    for (int c = 0; c < 3; c++) p[c] = P->origin[c] + P->h * (double)P->pp[3 * idx + c];
    if (pp_index) *pp_index = idx;
}

/* ------------------------------------------------------------------ trilinear lookup */
static double node(const or_pocket *P, const float *grid, int i, int j, int k) {
    return (double)grid[((size_t)k * P->n + j) * P->n + i];
}

static double lerp(double a, double b, double t) { return a + t * (b - a); }

/* Clamp a position into the grid box. */
void or_clamp_box(const or_pocket *P, const double x[3], double xhat[3]) {
    for (int c = 0; c < 3; c++) {
        double lo = P->origin[c], hi = P->origin[c] + P->h * (P->n - 1);
        xhat[c] = x[c] < lo ? lo : (x[c] > hi ? hi : x[c]);
    }
}

double or_trilinear(const or_pocket *P, const float *grid, const double x[3]) {
    double xh[3];
    or_clamp_box(P, x, xh);
    int i0[3];
    double f[3];
    for (int c = 0; c < 3; c++) {
        double g = (xh[c] - P->origin[c]) / P->h;
        int fl = (int)floor(g);
        if (fl > P->n - 2) fl = P->n - 2;
        if (fl < 0) fl = 0;
        i0[c] = fl;
        f[c] = g - fl;
    }
    int i = i0[0], j = i0[1], k = i0[2];
    double c00 = lerp(node(P, grid, i, j, k), node(P, grid, i + 1, j, k), f[0]);
    double c10 = lerp(node(P, grid, i, j + 1, k), node(P, grid, i + 1, j + 1, k), f[0]);
    double c01 = lerp(node(P, grid, i, j, k + 1), node(P, grid, i + 1, j, k + 1), f[0]);
    double c11 = lerp(node(P, grid, i, j + 1, k + 1), node(P, grid, i + 1, j + 1, k + 1), f[0]);
    double c0 = lerp(c00, c10, f[1]);
    double c1 = lerp(c01, c11, f[1]);
    return lerp(c0, c1, f[2]);
}

/* ------------------------------------------------------------------ torsion rotation
 * Rodrigues' formula: turn x by theta (cos c, sin s) about the unit axis
 * u = (xb - xa)/|xb - xa| through xb, right-hand rule. */
void or_rotate_about(const double xa[3], const double xb[3], double c, double s, const double x[3],
                     double out[3]) {
    double u[3] = {xb[0] - xa[0], xb[1] - xa[1], xb[2] - xa[2]};
    double nu = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    u[0] /= nu; u[1] /= nu; u[2] /= nu;
    double v[3] = {x[0] - xb[0], x[1] - xb[1], x[2] - xb[2]};
    double uv = u[0] * v[0] + u[1] * v[1] + u[2] * v[2];
    double cr[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
    for (int d = 0; d < 3; d++) out[d] = xb[d] + v[d] * c + cr[d] * s + u[d] * uv * (1.0 - c);
}

/* ------------------------------------------------------------------ pose energy */
double or_atom_energy(const or_pocket *P, const double x[3], double q, int type) {
    double xh[3];
    or_clamp_box(P, x, xh);
    double dx = x[0] - xh[0], dy = x[1] - xh[1], dz = x[2] - xh[2];
    double out = sqrt(dx * dx + dy * dy + dz * dz);
    return P->type_w[type] * or_trilinear(P, P->phi_v, xh) + q * or_trilinear(P, P->phi_e, xh) +
           P->k_out * out;
}

double or_pose_energy(const or_pocket *P, int32_t N, const double *xyz, const float *q, const uint8_t *type,
                      double *eabs) {
    double E = 0.0, A = 0.0;
    for (int i = 0; i < N; i++) {
        double e = or_atom_energy(P, xyz + 3 * i, (double)q[i], type[i]);
        E += e;
        A += fabs(e);
    }
    if (eabs) *eabs = A;
    return E;
}

/* ------------------------------------------------------------------ topology */
/* Checks the depth-first preorder layout and fills end[i] = one past the last
 * atom of subtree(i).  Returns 0 when valid. */
int or_topology(int32_t N, const int16_t *parent, int32_t *end) {
    if (N < 1 || N > OR_MAXN || parent[0] != -1) return -1;
    for (int i = 1; i < N; i++) {
        int p = parent[i];
        if (p < 0 || p >= i) return -1;
        /* preorder: the parent of i is i-1 or one of i-1's ancestors */
        int v = i - 1;
        while (v != p && v >= 0) v = (v == 0) ? -1 : parent[v];
        if (v != p) return -1;
    }
    for (int i = 0; i < N; i++) end[i] = i + 1;
    for (int i = N - 1; i >= 1; i--)
        if (end[i] > end[parent[i]]) end[parent[i]] = end[i];
    return 0;
}

int or_validate(int32_t N, const int16_t *parent, const uint8_t *type, int32_t R, const int16_t *rot_child,
                int32_t *end) {
    if (or_topology(N, parent, end) != 0) return -1;
    for (int i = 0; i < N; i++)
        if (type[i] > 4) return -1;
    if (R < 0) return -1;
    for (int k = 0; k < R; k++) {
        if (rot_child[k] < 1 || rot_child[k] >= N) return -1;
        if (k > 0 && rot_child[k] <= rot_child[k - 1]) return -1;
    }
    return 0;
}

/* ------------------------------------------------------------------ ranking */
/* Rank the S final poses (poses[S][N][3]) of a ligand and rescore the first K.
 * Outputs: G[S] geometric scores, order[S] ranked restarts, leader[S] cluster
 * leader of each restart (the restart itself when it leads), best_r/best_E. */
void or_rank_poses(const or_pocket *P, int32_t S, int32_t N, const double *poses, const double *E, double thr,
                   int32_t K, double *G, int32_t *order, int32_t *leader, int32_t *best_r, double *best_E) {
    for (int r = 0; r < S; r++) {
        double g = 0.0;
        for (int i = 0; i < N; i++) g += or_trilinear(P, P->phi_o, poses + ((size_t)r * N + i) * 3);
        G[r] = g;
    }
    /* geometric order: higher G first, lower restart on ties (insertion sort) */
    int32_t *geo = (int32_t *)malloc(sizeof(int32_t) * S);
    for (int r = 0; r < S; r++) {
        int p = r;
        while (p > 0 && G[geo[p - 1]] < G[r]) { geo[p] = geo[p - 1]; p--; }
        geo[p] = r;
    }
    /* greedy leader clustering in geometric order */
    int32_t *leads = (int32_t *)malloc(sizeof(int32_t) * S);
    int nl = 0;
    for (int p = 0; p < S; p++) {
        const int r = geo[p];
        leader[r] = r;
        if (thr > 0.0) {
            for (int k = 0; k < nl; k++) {
                const int q = leads[k];
                double ss = 0.0;
                for (int i = 0; i < N; i++)
                    for (int c = 0; c < 3; c++) {
                        const double d = poses[((size_t)r * N + i) * 3 + c] - poses[((size_t)q * N + i) * 3 + c];
                        ss += d * d;
                    }
                if (ss / N <= thr * thr) { leader[r] = q; break; }
            }
        }
        if (leader[r] == r) leads[nl++] = r;
    }
    /* ranking: leaders in geometric order, then the others */
    int n = 0;
    for (int p = 0; p < S; p++) if (leader[geo[p]] == geo[p]) order[n++] = geo[p];
    for (int p = 0; p < S; p++) if (leader[geo[p]] != geo[p]) order[n++] = geo[p];
    /* rescore the first K */
    const int k = (K <= 0 || K > S) ? S : K;
    int br = -1;
    double be = INFINITY;
    for (int p = 0; p < k; p++) {
        const int r = order[p];
        if (E[r] < be || (E[r] == be && r < br)) { be = E[r]; br = r; }
    }
    *best_r = br;
    *best_E = be;
    free(geo);
    free(leads);
}

/* ------------------------------------------------------------------ rigid moves */
#define OR_RIGID_CANDIDATES 13

/* Candidate `cand` of a rigid move (see "rigid" above) applied to N atoms. */
void or_rigid_candidate(int32_t N, const double *X, int32_t cand, double shift, double angle, double *out) {
    double c[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < N; i++)
        for (int d = 0; d < 3; d++) c[d] += X[3 * i + d];
    for (int d = 0; d < 3; d++) c[d] /= N;
    for (int i = 0; i < N; i++) {
        const double *x = X + 3 * i;
        double *o = out + 3 * i;
        o[0] = x[0]; o[1] = x[1]; o[2] = x[2];
        if (cand >= 1 && cand <= 6) {
            const int ax = (cand - 1) / 2;
            o[ax] += (cand % 2 == 1) ? shift : -shift;
        } else if (cand >= 7 && cand <= 12) {
            const int ax = (cand - 7) / 2;
            const double th = (cand % 2 == 1) ? angle : -angle, cs = cos(th), sn = sin(th);
            const int j = (ax + 1) % 3, k = (ax + 2) % 3; /* (x: y, z), (y: z, x), (z: x, y) */
            const double vj = x[j] - c[j], vk = x[k] - c[k];
            o[j] = c[j] + cs * vj - sn * vk;
            o[k] = c[k] + sn * vj + cs * vk;
        }
    }
}

static double or_geometric_score(const or_pocket *P, int32_t N, const double *X) {
    double g = 0.0;
    for (int i = 0; i < N; i++) g += or_trilinear(P, P->phi_o, X + 3 * i);
    return g;
}

/* ------------------------------------------------------------------ docking */
/* Outputs (any may be NULL except restart_E):
 *   restart_E[S], restart_Eabs[S]      score and sum of |per-atom terms| per restart
 *   choice[S][P][R]                    step applied at each decision
 *   own[S][P][R]                       the oracle's own argmax at that decision
 *   trace_s[S][P][R][A], trace_d2[...] overlap score and min clash distance^2 per step
 *                                      (+inf when the bond has no checked pair)
 *   poses[S][N][3]                     final pose of every restart
 *   best_pose[N][3]                    final pose of the best restart
 *   rank_out[2S] (with ranking)        ranked restarts, then each restart's leader
 *   geo_out[S] (with ranking)          geometric score of every restart
 *   choice_rigid / own_rigid[S][P][rigid_steps], trace_G[...][13]: rigid
 *                                      moves applied / chosen by the oracle,
 *                                      and every candidate's geometric score
 * replay_rigid (optional): apply these rigid moves instead.
 * replay[S][P][R] (optional): apply these steps instead of the oracle's own,
 * still recording what the oracle would have chosen. */
int or_dock_ligand(const or_pocket *P, const or_params *prm, int32_t N, const float *x, const float *y,
                   const float *z, const float *q, const uint8_t *type, const int16_t *parent, int32_t R,
                   const int16_t *rot_child, uint64_t uid, const uint8_t *replay, double *restart_E,
                   double *restart_Eabs, uint8_t *choice, uint8_t *own, double *trace_s, double *trace_d2,
                   double *poses, double *best_pose, int32_t *best_r, double *best_E, int32_t *rank_out,
                   double *geo_out, const uint8_t *replay_rigid, uint8_t *choice_rigid, uint8_t *own_rigid,
                   double *trace_G) {
    int32_t end[OR_MAXN];
    if (or_validate(N, parent, type, R, rot_child, end) != 0) return -1;
    const int S = prm->restarts, PS = prm->passes, A = prm->angle_steps;
    if (S < 1 || PS < 0 || A < 1 || A > 255 || P->n_pp < 1 || P->n < 2) return -1;

    double cen[3] = {0, 0, 0};
    for (int i = 0; i < N; i++) { cen[0] += x[i]; cen[1] += y[i]; cen[2] += z[i]; }
    for (int c = 0; c < 3; c++) cen[c] /= N;

    double X[OR_MAXN][3], T[OR_MAXN][3];
    double bestE = INFINITY;
    int bestR = -1;
    const double dc2 = prm->d_clash * prm->d_clash;
    const int ranking = prm->cluster_rmsd > 0.0 || (prm->rescore_top > 0 && prm->rescore_top < S);
    double *allposes = ranking ? (double *)malloc(sizeof(double) * 3 * (size_t)S * N) : NULL;

    for (int r = 0; r < S; r++) {
        double Rm[9], p[3];
        or_restart_pose(P, prm, uid, r, Rm, p, NULL);
        for (int i = 0; i < N; i++) {
            double v[3] = {x[i] - cen[0], y[i] - cen[1], z[i] - cen[2]};
            for (int c = 0; c < 3; c++) X[i][c] = Rm[3 * c] * v[0] + Rm[3 * c + 1] * v[1] + Rm[3 * c + 2] * v[2] + p[c];
        }
        for (int ps = 0; ps < PS; ps++) {
            for (int k = 0; k < R; k++) {
                const int b = rot_child[k], a = parent[b], e = end[b];
                const size_t dec = ((size_t)r * PS + ps) * R + k;
                int own_t = 0;
                double own_s = -INFINITY;
                for (int t = 0; t < A; t++) {
                    double th = 2.0 * M_PI * t / A, c = cos(th), s = sin(th);
                    for (int i = b + 1; i < e; i++) {
                        if (t == 0) memcpy(T[i], X[i], sizeof(T[i]));
                        else or_rotate_about(X[a], X[b], c, s, X[i], T[i]);
                    }
                    double sc = 0.0;
                    for (int i = b + 1; i < e; i++) sc += or_trilinear(P, P->phi_o, T[i]);
                    double d2min = INFINITY;
                    for (int i = b + 1; i < e; i++)
                        for (int j = 0; j < N; j++) {
                            if (j >= b && j < e) continue;              /* j in subtree(b): not fixed */
                            if (j == a && parent[i] == b) continue;     /* 1-3 pair through the bond */
                            double dx = T[i][0] - X[j][0], dy = T[i][1] - X[j][1], dz = T[i][2] - X[j][2];
                            double d2 = dx * dx + dy * dy + dz * dz;
                            if (d2 < d2min) d2min = d2;
                        }
                    if (trace_s) trace_s[dec * A + t] = sc;
                    if (trace_d2) trace_d2[dec * A + t] = d2min;
                    int admissible = (t == 0) || (d2min >= dc2);
                    if (admissible && sc > own_s) { own_s = sc; own_t = t; }
                }
                int ch = replay ? replay[dec] : own_t;
                if (ch < 0 || ch >= A) return -2;
                if (own) own[dec] = (uint8_t)own_t;
                if (choice) choice[dec] = (uint8_t)ch;
                if (ch != 0) {
                    double th = 2.0 * M_PI * ch / A, c = cos(th), s = sin(th);
                    double xa[3] = {X[a][0], X[a][1], X[a][2]}, xb[3] = {X[b][0], X[b][1], X[b][2]};
                    for (int i = b + 1; i < e; i++) {
                        double o[3];
                        or_rotate_about(xa, xb, c, s, X[i], o);
                        memcpy(X[i], o, sizeof(o));
                    }
                }
            }
            /* rigid greedy moves of the whole ligand */
            for (int j = 0; j < prm->rigid_steps; j++) {
                const size_t dec = ((size_t)r * PS + ps) * prm->rigid_steps + j;
                int own_c = 0;
                double own_g = -INFINITY;
                for (int cand = 0; cand < OR_RIGID_CANDIDATES; cand++) {
                    or_rigid_candidate(N, &X[0][0], cand, prm->rigid_shift, 2.0 * M_PI / A, &T[0][0]);
                    double g = or_geometric_score(P, N, &T[0][0]);
                    if (trace_G) trace_G[dec * OR_RIGID_CANDIDATES + cand] = g;
                    if (g > own_g) { own_g = g; own_c = cand; }
                }
                int ch = replay_rigid ? replay_rigid[dec] : own_c;
                if (ch < 0 || ch >= OR_RIGID_CANDIDATES) return -2;
                if (own_rigid) own_rigid[dec] = (uint8_t)own_c;
                if (choice_rigid) choice_rigid[dec] = (uint8_t)ch;
                if (ch != 0) {
                    or_rigid_candidate(N, &X[0][0], ch, prm->rigid_shift, 2.0 * M_PI / A, &T[0][0]);
                    memcpy(X, T, sizeof(double) * 3 * N);
                }
            }
        }
        double eabs;
        double E = or_pose_energy(P, N, &X[0][0], q, type, &eabs);
        restart_E[r] = E;
        if (restart_Eabs) restart_Eabs[r] = eabs;
        if (poses) memcpy(poses + (size_t)r * N * 3, &X[0][0], sizeof(double) * 3 * N);
        if (allposes) memcpy(allposes + (size_t)r * N * 3, &X[0][0], sizeof(double) * 3 * N);
        if (E < bestE) {
            bestE = E;
            bestR = r;
            if (best_pose) memcpy(best_pose, &X[0][0], sizeof(double) * 3 * N);
        }
    }
    if (ranking) {
        double *G = (double *)malloc(sizeof(double) * S);
        int32_t *ord = (int32_t *)malloc(sizeof(int32_t) * S), *lead = (int32_t *)malloc(sizeof(int32_t) * S);
        or_rank_poses(P, S, N, allposes, restart_E, prm->cluster_rmsd, prm->rescore_top, G, ord, lead, &bestR,
                      &bestE);
        if (rank_out) {
            memcpy(rank_out, ord, sizeof(int32_t) * S);
            memcpy(rank_out + S, lead, sizeof(int32_t) * S);
        }
        if (geo_out) memcpy(geo_out, G, sizeof(double) * S);
        if (best_pose && bestR >= 0) memcpy(best_pose, allposes + (size_t)bestR * N * 3, sizeof(double) * 3 * N);
        free(G);
        free(ord);
        free(lead);
        free(allposes);
    }
    if (best_r) *best_r = bestR;
    if (best_E) *best_E = bestE;
    return 0;
}

/* Batch in CSR layout (see the generator for the layout).  Per-ligand output
 * offsets: restart arrays l*S; decisions S*P*rot_off[l]; traces A*S*P*rot_off[l];
 * poses 3*S*atom_off[l]; best poses 3*atom_off[l]; rankings 2*S*l; geometric
 * scores S*l; rigid decisions S*P*rigid_steps*l (traces 13 times that).
 * status[l] = 0 or -1. */
int or_dock_batch(const or_pocket *P, const or_params *prm, int32_t L, const int32_t *atom_off, const float *x,
                  const float *y, const float *z, const float *q, const uint8_t *type, const int16_t *parent,
                  const int32_t *rot_off, const int16_t *rot_child, const uint64_t *uid, const uint8_t *replay,
                  double *restart_E, double *restart_Eabs, uint8_t *choice, uint8_t *own, double *trace_s,
                  double *trace_d2, double *poses, double *best_pose, int32_t *best_r, double *best_E,
                  int32_t *status, int32_t *rank_out, double *geo_out, const uint8_t *replay_rigid,
                  uint8_t *choice_rigid, uint8_t *own_rigid, double *trace_G, int32_t nthreads) {
    const int S = prm->restarts, PS = prm->passes, A = prm->angle_steps;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1) reduction(+ : bad)
    for (int l = 0; l < L; l++) {
        const int a0 = atom_off[l], N = atom_off[l + 1] - a0;
        const int r0 = rot_off[l], Rl = rot_off[l + 1] - r0;
        const size_t d0 = (size_t)S * PS * r0;
        const size_t rd0 = (size_t)S * PS * prm->rigid_steps * l;
        int rc = or_dock_ligand(
            P, prm, N, x + a0, y + a0, z + a0, q + a0, type + a0, parent + a0, Rl, rot_child + r0, uid[l],
            replay ? replay + d0 : NULL, restart_E + (size_t)l * S, restart_Eabs ? restart_Eabs + (size_t)l * S : NULL,
            choice ? choice + d0 : NULL, own ? own + d0 : NULL, trace_s ? trace_s + d0 * A : NULL,
            trace_d2 ? trace_d2 + d0 * A : NULL, poses ? poses + (size_t)3 * S * a0 : NULL,
            best_pose ? best_pose + (size_t)3 * a0 : NULL, best_r + l, best_E + l,
            rank_out ? rank_out + (size_t)2 * S * l : NULL, geo_out ? geo_out + (size_t)S * l : NULL,
            replay_rigid ? replay_rigid + rd0 : NULL, choice_rigid ? choice_rigid + rd0 : NULL,
            own_rigid ? own_rigid + rd0 : NULL, trace_G ? trace_G + rd0 * OR_RIGID_CANDIDATES : NULL);
        status[l] = rc;
        if (rc != 0) bad++;
    }
    return bad;
}

/* Energies of given poses (no docking): poses in CSR layout, xyz interleaved. */
void or_score_poses(const or_pocket *P, int32_t L, const int32_t *atom_off, const double *xyz, const float *q,
                    const uint8_t *type, double *E, double *Eabs) {
    for (int l = 0; l < L; l++) {
        int a0 = atom_off[l], N = atom_off[l + 1] - a0;
        E[l] = or_pose_energy(P, N, xyz + 3 * (size_t)a0, q + a0, type + a0, Eabs ? Eabs + l : NULL);
    }
}

/* ------------------------------------------------------------------ flattening
 * Ligand pre-processing (Sec. 3.1, step 1; protein independent): the torsional
 * bonds are turned to maximise the sum of the distances between all atom
 * pairs.  Reading: the greedy sweep of the docking step with this objective in
 * place of the overlap score -- for pass = 0..P-1 and torsional bond k in
 * ascending child order, step t = 0..A-1 turns the moving set about the bond
 * axis as in the sweep; D(t) = sum over all pairs i < j of |x_i - x_j|; the
 * admissible step (the sweep's clash rule) with the largest D is applied, the
 * lowest step on ties.  The ligand stays in its input frame.
 * Outputs: xyz_out[N][3]; choice/own[P][R]; trace_D/trace_d2[P][R][A] (D and
 * the minimum clash distance^2 of every step, +inf without checked pairs);
 * D_out = D of the final conformation.  replay[P][R] (optional) applies the
 * given steps instead, still recording the oracle's own choices. */
static double or_pair_distance_sum(int32_t N, double (*T)[3]) {
    double D = 0.0;
    for (int i = 0; i < N; i++)
        for (int j = i + 1; j < N; j++) {
            double dx = T[i][0] - T[j][0], dy = T[i][1] - T[j][1], dz = T[i][2] - T[j][2];
            D += sqrt(dx * dx + dy * dy + dz * dz);
        }
    return D;
}

int or_flatten_ligand(int32_t N, const float *x, const float *y, const float *z, const uint8_t *type,
                      const int16_t *parent, int32_t R, const int16_t *rot_child, int32_t passes, int32_t A,
                      double d_clash, const uint8_t *replay, double *xyz_out, uint8_t *choice, uint8_t *own,
                      double *trace_D, double *trace_d2, double *D_out) {
    int32_t end[OR_MAXN];
    if (or_validate(N, parent, type, R, rot_child, end) != 0) return -1;
    if (passes < 0 || A < 1 || A > 255) return -1;
    double X[OR_MAXN][3], T[OR_MAXN][3];
    for (int i = 0; i < N; i++) { X[i][0] = x[i]; X[i][1] = y[i]; X[i][2] = z[i]; }
    const double dc2 = d_clash * d_clash;
    for (int ps = 0; ps < passes; ps++) {
        for (int k = 0; k < R; k++) {
            const int b = rot_child[k], a = parent[b], e = end[b];
            const size_t dec = (size_t)ps * R + k;
            int own_t = 0;
            double own_D = -INFINITY;
            for (int t = 0; t < A; t++) {
                double th = 2.0 * M_PI * t / A, c = cos(th), s = sin(th);
                memcpy(T, X, sizeof(double) * 3 * N);
                if (t != 0)
                    for (int i = b + 1; i < e; i++) or_rotate_about(X[a], X[b], c, s, X[i], T[i]);
                double D = or_pair_distance_sum(N, T);
                double d2min = INFINITY;
                for (int i = b + 1; i < e; i++)
                    for (int j = 0; j < N; j++) {
                        if (j >= b && j < e) continue;
                        if (j == a && parent[i] == b) continue;
                        double dx = T[i][0] - T[j][0], dy = T[i][1] - T[j][1], dz = T[i][2] - T[j][2];
                        double d2 = dx * dx + dy * dy + dz * dz;
                        if (d2 < d2min) d2min = d2;
                    }
                if (trace_D) trace_D[dec * A + t] = D;
                if (trace_d2) trace_d2[dec * A + t] = d2min;
                int admissible = (t == 0) || (d2min >= dc2);
                if (admissible && D > own_D) { own_D = D; own_t = t; }
            }
            int ch = replay ? replay[dec] : own_t;
            if (ch < 0 || ch >= A) return -2;
            if (own) own[dec] = (uint8_t)own_t;
            if (choice) choice[dec] = (uint8_t)ch;
            if (ch != 0) {
                double th = 2.0 * M_PI * ch / A, c = cos(th), s = sin(th);
                double xa[3] = {X[a][0], X[a][1], X[a][2]}, xb[3] = {X[b][0], X[b][1], X[b][2]};
                for (int i = b + 1; i < e; i++) {
                    double o[3];
                    or_rotate_about(xa, xb, c, s, X[i], o);
                    memcpy(X[i], o, sizeof(o));
                }
            }
        }
    }
    if (xyz_out) memcpy(xyz_out, X, sizeof(double) * 3 * N);
    if (D_out) *D_out = or_pair_distance_sum(N, X);
    return 0;
}

/* Batch in CSR layout.  Per-ligand offsets: xyz 3*atom_off[l]; decisions
 * P*rot_off[l]; traces A*P*rot_off[l]; D l.  status[l] = 0 or -1. */
int or_flatten_batch(int32_t L, const int32_t *atom_off, const float *x, const float *y, const float *z,
                     const uint8_t *type, const int16_t *parent, const int32_t *rot_off, const int16_t *rot_child,
                     int32_t passes, int32_t A, double d_clash, const uint8_t *replay, double *xyz_out,
                     uint8_t *choice, uint8_t *own, double *trace_D, double *trace_d2, double *D_out,
                     int32_t *status, int32_t nthreads) {
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1) reduction(+ : bad)
    for (int l = 0; l < L; l++) {
        const int a0 = atom_off[l], N = atom_off[l + 1] - a0;
        const int r0 = rot_off[l], Rl = rot_off[l + 1] - r0;
        const size_t d0 = (size_t)passes * r0;
        int rc = or_flatten_ligand(N, x + a0, y + a0, z + a0, type + a0, parent + a0, Rl, rot_child + r0, passes, A,
                                   d_clash, replay ? replay + d0 : NULL, xyz_out ? xyz_out + (size_t)3 * a0 : NULL,
                                   choice ? choice + d0 : NULL, own ? own + d0 : NULL,
                                   trace_D ? trace_D + d0 * A : NULL, trace_d2 ? trace_d2 + d0 * A : NULL,
                                   D_out ? D_out + l : NULL);
        status[l] = rc;
        if (rc != 0) bad++;
    }
    return bad;
}
