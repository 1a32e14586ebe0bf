// Docking kernels for sm_103a (GB300).
//
// The dock-and-score step of the paper (Sec. 3.1) on the GPU.  One CTA docks
// one ligand: its warps share the ligand's topology in shared memory and each
// warp runs one restart at a time (restarts are tiled over the CTA's warps).
//
// Inside a warp the 36 torsion steps of a bond map onto lanes: lane t owns
// step t (steps 32..35 are spread over the warp in a short tail loop), so the
// per-step overlap sums need no cross-lane reduction and the choice of step is
// a 5-level shuffle argmax.  Moving atoms are processed in bundles of 32 (the
// paper's CUDA design also works in bundles of 32 atoms, Sec. 3.1): each lane
// builds the circle one atom traces about the bond axis,
//     x(theta) = p + e1 cos(theta) + e2 sin(theta),
// and every lane evaluates its own step on that circle with two FMAs per
// coordinate, then reads one 32-byte cell of trilinear coefficients of the
// overlap grid (L2-resident, read-only path).
//
// The clash test uses the same circles: for a moving atom i and a fixed atom j
//     |x_i(theta) - x_j|^2 = C + 2a cos(theta) + 2b sin(theta),
//     C = |p - x_j|^2 + |e1|^2,  a = (p - x_j).e1,  b = (p - x_j).e2,
// whose minimum over the circle is C - 2 sqrt(a^2 + b^2).  Pairs whose minimum
// stays above d_clash^2 can never clash and are dropped with one test; the few
// others are evaluated for all 36 steps at once (lanes = steps), so every
// decision gets its full admissibility mask in one pass.
//
// Positions live in centred grid units (see lg_internal.h).
#include <curand_philox4x32_x.h>

#include "lg_internal.h"

namespace lg {

#define LG_FULL 0xffffffffu

__constant__ float c_cos[LG_ANGLE_STEPS];
__constant__ float c_sin[LG_ANGLE_STEPS];

void set_angle_tables(const float *cosv, const float *sinv) {
    cudaMemcpyToSymbol(c_cos, cosv, sizeof(float) * LG_ANGLE_STEPS);
    cudaMemcpyToSymbol(c_sin, sinv, sizeof(float) * LG_ANGLE_STEPS);
}

// ------------------------------------------------------------------ Philox4x32-10
// Salmon, Moraes, Dror, Shaw, SC'11: ten rounds; each multiplies words 0 and 2
// by the round constants, keeps both halves of the products, mixes the high
// halves with the other two words and the key; the key advances by the two
// Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; r++) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// ------------------------------------------------------------------ grid lookups
// Floor of an index-space coordinate in [0, 2^22) by adding 1.5*2^23 with
// round-down: the integer part lands in the low mantissa bits of t and
// t - 1.5*2^23 is exact, as is the fraction g - floor(g).
constexpr float kMagic = 12582912.0f;  // bit pattern 0x4B400000

__device__ __forceinline__ float floor_frac(float g, float &t) {
    t = __fadd_rd(g, kMagic);
    return g - (t - kMagic);
}

// Flat cell index (k*n + j)*n + i from the three round-down sums (32-bit
// wrap-around arithmetic; the true result is small and non-negative).
__device__ __forceinline__ uint32_t cell_index(float tx, float ty, float tz, uint32_t n, uint32_t n2, uint32_t moff) {
    return __float_as_uint(tz) * n2 + __float_as_uint(ty) * n + __float_as_uint(tx) - moff;
}

// Trilinear polynomial of one cell: lo = (c0, c1, c2, c3), hi = (c4, c5, c6, c7).
__device__ __forceinline__ float cell_eval(const float4 lo, const float4 hi, float fx, float fy, float fz) {
    const float t1 = fmaf(fz, hi.w, hi.x);  // c4 + c7 fz
    const float t2 = fmaf(fz, hi.y, lo.y);  // c1 + c5 fz
    const float ax = fmaf(fy, t1, t2);      // d p / d fx
    const float t4 = fmaf(fz, hi.z, lo.z);  // c2 + c6 fz
    const float t5 = fmaf(fz, lo.w, lo.x);  // c0 + c3 fz
    const float b = fmaf(fy, t4, t5);
    return fmaf(fx, ax, b);
}

__device__ __forceinline__ float clampg(float g, float gmax) { return fminf(fmaxf(g, 0.0f), gmax); }

struct GridK {  // lookup constants of a pocket
    const float4 *cells;
    uint32_t n, n2, moff;
    float gmax;
};

__device__ __forceinline__ GridK grid_k(const PocketDev &P, const float4 *cells) {
    GridK g;
    g.cells = cells;
    g.n = (uint32_t)P.n;
    g.n2 = g.n * g.n;
    g.moff = 0x4B400000u * (g.n2 + g.n + 1u);
    g.gmax = P.gmax;
    return g;
}

// Overlap-field value at an index-space point known to lie in [0, n-1]^3.
__device__ __forceinline__ float lookup_in(const GridK &G, float gx, float gy, float gz) {
    float tx, ty, tz;
    const float fx = floor_frac(gx, tx), fy = floor_frac(gy, ty), fz = floor_frac(gz, tz);
    const float4 *p = G.cells + 2 * (size_t)cell_index(tx, ty, tz, G.n, G.n2, G.moff);
    const float4 lo = __ldg(p), hi = __ldg(p + 1);
    return cell_eval(lo, hi, fx, fy, fz);
}

// Overlap-field value at any index-space point (clamped to the box).
__device__ __forceinline__ float lookup_clamped(const GridK &G, float gx, float gy, float gz) {
    return lookup_in(G, clampg(gx, G.gmax), clampg(gy, G.gmax), clampg(gz, G.gmax));
}

// Per-atom energy term at a centred-grid-unit position: type weight * vdW grid
// + charge * electrostatic grid at the clamped position, plus k_out times the
// distance (A) outside the box.
__device__ __forceinline__ float atom_energy(const PocketDev &P, const GridK &G, float x, float y, float z, float w,
                                             float q) {
    const float gx = x + P.c0, gy = y + P.c0, gz = z + P.c0;
    const float cx = clampg(gx, P.gmax), cy = clampg(gy, P.gmax), cz = clampg(gz, P.gmax);
    const float dx = gx - cx, dy = gy - cy, dz = gz - cz;
    const float out = P.h * sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
    float tx, ty, tz;
    const float fx = floor_frac(cx, tx), fy = floor_frac(cy, ty), fz = floor_frac(cz, tz);
    const float4 *p = G.cells + 4 * (size_t)cell_index(tx, ty, tz, G.n, G.n2, G.moff);
    const float v = cell_eval(__ldg(p), __ldg(p + 1), fx, fy, fz);
    const float e = cell_eval(__ldg(p + 2), __ldg(p + 3), fx, fy, fz);
    return fmaf(w, v, fmaf(q, e, P.k_out * out));
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(LG_FULL, v, o);
    return v;
}

// ------------------------------------------------------------------ shared-memory views
struct CtaView {
    float4 *dv;
    double *wE;
    float *d0x, *d0y, *d0z;
    float2 *wq;
    int *par, *rch, *rend, *wR;
};

struct WarpView {
    float4 *bundle;  // 32 atoms x 4 float4 (see sweep_bond)
    float4 *axis;
    float *Xx, *Xy, *Xz;
    float *Bx, *By, *Bz;
    uint8_t *tcur, *tbest;
};

__device__ __forceinline__ CtaView cta_view(char *sm, const Layout &L) {
    CtaView v;
    v.dv = (float4 *)(sm + L.o_dv);
    v.wE = (double *)(sm + L.o_wE);
    v.d0x = (float *)(sm + L.o_d0);
    v.d0y = v.d0x + L.nmax;
    v.d0z = v.d0y + L.nmax;
    v.wq = (float2 *)(sm + L.o_wq);
    v.par = (int *)(sm + L.o_par);
    v.rch = (int *)(sm + L.o_rch);
    v.rend = (int *)(sm + L.o_rend);
    v.wR = (int *)(sm + L.o_wR);
    return v;
}

__device__ __forceinline__ WarpView warp_view(char *sm, const Layout &L, int w) {
    char *b = sm + L.cta_bytes + w * L.warp_bytes;
    WarpView v;
    v.bundle = (float4 *)(b + L.o_bundle);
    v.axis = (float4 *)(b + L.o_axis);
    v.Xx = (float *)(b + L.o_X);
    v.Xy = v.Xx + L.nmax;
    v.Xz = v.Xy + L.nmax;
    v.Bx = (float *)(b + L.o_best);
    v.By = v.Bx + L.nmax;
    v.Bz = v.By + L.nmax;
    v.tcur = (uint8_t *)(b + L.o_tcur);
    v.tbest = (uint8_t *)(b + L.o_tbest);
    return v;
}

// ------------------------------------------------------------------ one torsion decision
// Sweeps torsional bond k of the pose held by this warp, applies the chosen
// step and returns it (0..35).  lane owns step `lane` (cos cl, sin sl) and, in
// the tail, step 32 + (lane & 3) (cos ct, sin st).
//
// Bundle entry of a moving atom (index space = centred grid units + c0):
//   q0 = (P.x, P.y, P.z, e1.x)      P = circle centre in index space
//   q1 = (e1.y, e1.z, e2.x, e2.y)
//   q2 = (e2.z, |e1|^2, inside, 0)  inside = 1 when the whole circle is in the box
//   q3 = (p.x, p.y, p.z, 0)         p = circle centre in centred grid units
__device__ int sweep_bond(const DockArgs &A, const GridK &G, const CtaView &cv, const WarpView &wv, int N, int R,
                          int k, int lane, float cl, float sl, float ct, float st) {
    const int b = cv.rch[k], a = cv.par[b], e = cv.rend[k];
    const int m = e - b - 1;
    if (m <= 0) return 0;  // nothing moves: every step scores 0, step 0 wins

    const float xbx = wv.Xx[b], xby = wv.Xy[b], xbz = wv.Xz[b];
    const float4 ax = wv.axis[k];
    const float inv = rnorm3df(ax.x, ax.y, ax.z);
    const float ux = ax.x * inv, uy = ax.y * inv, uz = ax.z * inv;
    const float c0 = A.pocket.c0, lim = G.gmax - 1e-3f;
    const float dc2 = A.dc2g;
    const int nF = N - (e - b);  // atoms outside subtree(b): [0, b) and [e, N)

    float acc = 0.0f, acc_t = 0.0f;
    bool clash_lo = false, clash_hi = false;
    for (int base = b + 1; base < e; base += 32) {
        const int cnt = min(32, e - base);
        if (lane < cnt) {
            const int i = base + lane;
            const float dx = wv.Xx[i] - xbx, dy = wv.Xy[i] - xby, dz = wv.Xz[i] - xbz;
            const float w = fmaf(ux, dx, fmaf(uy, dy, uz * dz));
            const float px = fmaf(w, ux, xbx), py = fmaf(w, uy, xby), pz = fmaf(w, uz, xbz);
            const float e1x = fmaf(-w, ux, dx), e1y = fmaf(-w, uy, dy), e1z = fmaf(-w, uz, dz);
            const float e2x = fmaf(uy, dz, -uz * dy), e2y = fmaf(uz, dx, -ux * dz), e2z = fmaf(ux, dy, -uy * dx);
            const float Px = px + c0, Py = py + c0, Pz = pz + c0;
            const float rx = fabsf(e1x) + fabsf(e2x), ry = fabsf(e1y) + fabsf(e2y), rz = fabsf(e1z) + fabsf(e2z);
            const bool inside = Px - rx >= 1e-3f && Px + rx <= lim && Py - ry >= 1e-3f && Py + ry <= lim &&
                                Pz - rz >= 1e-3f && Pz + rz <= lim;
            float4 *q = wv.bundle + 4 * lane;
            q[0] = make_float4(Px, Py, Pz, e1x);
            q[1] = make_float4(e1y, e1z, e2x, e2y);
            q[2] = make_float4(e2z, fmaf(e1x, e1x, fmaf(e1y, e1y, e1z * e1z)), inside ? 1.0f : 0.0f, 0.0f);
            q[3] = make_float4(px, py, pz, 0.0f);
        }
        __syncwarp();
        // steps 0..31: lane t scores step t for every atom of the bundle
#pragma unroll 4
        for (int t = 0; t < cnt; ++t) {
            const float4 q0 = wv.bundle[4 * t], q1 = wv.bundle[4 * t + 1], q2 = wv.bundle[4 * t + 2];
            const float gx = fmaf(q1.z, sl, fmaf(q0.w, cl, q0.x));
            const float gy = fmaf(q1.w, sl, fmaf(q1.x, cl, q0.y));
            const float gz = fmaf(q2.x, sl, fmaf(q1.y, cl, q0.z));
            acc += (q2.z != 0.0f) ? lookup_in(G, gx, gy, gz) : lookup_clamped(G, gx, gy, gz);
        }
        // steps 32..35: lane scores step 32 + (lane & 3) for atoms lane>>2, +8, ...
        for (int t = lane >> 2; t < cnt; t += 8) {
            const float4 q0 = wv.bundle[4 * t], q1 = wv.bundle[4 * t + 1], q2 = wv.bundle[4 * t + 2];
            const float gx = fmaf(q1.z, st, fmaf(q0.w, ct, q0.x));
            const float gy = fmaf(q1.w, st, fmaf(q1.x, ct, q0.y));
            const float gz = fmaf(q2.x, st, fmaf(q1.y, ct, q0.z));
            acc_t += lookup_clamped(G, gx, gy, gz);
        }
        // clash pairs (bundle atom ti, fixed atom jj), flattened over the warp
        const int npairs = cnt * nF;
        int ti = lane / nF, jj = lane - (lane / nF) * nF;
        for (int pb = 0; pb < npairs; pb += 32) {
            bool flag = false;
            float C = 0.0f, A2 = 0.0f, B2 = 0.0f;
            if (pb + lane < npairs) {
                const int j = jj < b ? jj : jj + (e - b);
                const float4 *q = wv.bundle + 4 * ti;
                const float4 q0 = q[0], q1 = q[1], q2 = q[2], q3 = q[3];
                const float wx = q3.x - wv.Xx[j], wy = q3.y - wv.Xy[j], wz = q3.z - wv.Xz[j];
                const float aa = fmaf(wx, q0.w, fmaf(wy, q1.x, wz * q1.y));
                const float bb = fmaf(wx, q1.z, fmaf(wy, q1.w, wz * q2.x));
                C = fmaf(wx, wx, fmaf(wy, wy, fmaf(wz, wz, q2.y)));
                const float T = C - dc2;
                const float s2 = fmaf(aa, aa, bb * bb);
                // the circle comes within d_clash of j iff T < 2 sqrt(a^2 + b^2)
                flag = (T <= 0.0f || T * T < 4.0004f * s2) && !(j == a && cv.par[base + ti] == b);
                A2 = 2.0f * aa;
                B2 = 2.0f * bb;
            }
            unsigned msk = __ballot_sync(LG_FULL, flag);
            while (msk) {
                const int src = __ffs(msk) - 1;
                msk &= msk - 1;
                const float Cs = __shfl_sync(LG_FULL, C, src);
                const float As = __shfl_sync(LG_FULL, A2, src);
                const float Bs = __shfl_sync(LG_FULL, B2, src);
                clash_lo |= fmaf(Bs, sl, fmaf(As, cl, Cs)) < dc2;
                clash_hi |= fmaf(Bs, st, fmaf(As, ct, Cs)) < dc2;
            }
            jj += 32;
            while (jj >= nF) {
                jj -= nF;
                ++ti;
            }
        }
        __syncwarp();
    }
    acc_t += __shfl_xor_sync(LG_FULL, acc_t, 4);
    acc_t += __shfl_xor_sync(LG_FULL, acc_t, 8);
    acc_t += __shfl_xor_sync(LG_FULL, acc_t, 16);
    if (lane == 0) clash_lo = false;  // step 0 (the current pose) is always admissible

    // highest-scoring admissible step, lowest step on ties
    float bs = clash_lo ? -INFINITY : acc;
    int ba = clash_lo ? 1024 : lane;
    if (lane < 4 && !clash_hi && acc_t > bs) {  // equal scores keep the lower step (lane < 32 + lane)
        bs = acc_t;
        ba = 32 + lane;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float os = __shfl_xor_sync(LG_FULL, bs, o);
        const int oa = __shfl_xor_sync(LG_FULL, ba, o);
        if (os > bs || (os == bs && oa < ba)) {
            bs = os;
            ba = oa;
        }
    }
    // every lane holds the same winner; take lane 0's so control flow stays
    // warp-uniform whatever the scores are
    const int t = __shfl_sync(LG_FULL, ba, 0);
    if (t <= 0 || t >= LG_ANGLE_STEPS) return 0;

    const float c = c_cos[t], s = c_sin[t];
    for (int i = b + 1 + lane; i < e; i += 32) {
        const float dx = wv.Xx[i] - xbx, dy = wv.Xy[i] - xby, dz = wv.Xz[i] - xbz;
        const float w = fmaf(ux, dx, fmaf(uy, dy, uz * dz));
        const float e1x = fmaf(-w, ux, dx), e1y = fmaf(-w, uy, dy), e1z = fmaf(-w, uz, dz);
        const float e2x = fmaf(uy, dz, -uz * dy), e2y = fmaf(uz, dx, -ux * dz), e2z = fmaf(ux, dy, -uy * dx);
        wv.Xx[i] = fmaf(e2x, s, fmaf(e1x, c, fmaf(w, ux, xbx)));
        wv.Xy[i] = fmaf(e2y, s, fmaf(e1y, c, fmaf(w, uy, xby)));
        wv.Xz[i] = fmaf(e2z, s, fmaf(e1z, c, fmaf(w, uz, xbz)));
    }
    // bond axes further down the subtree turn with it
    for (int kk = k + 1 + lane; kk < R; kk += 32) {
        if (cv.rch[kk] < e) {
            const float4 v = wv.axis[kk];
            const float uv = fmaf(ux, v.x, fmaf(uy, v.y, uz * v.z));
            const float cx = fmaf(uy, v.z, -uz * v.y), cy = fmaf(uz, v.x, -ux * v.z), cz = fmaf(ux, v.y, -uy * v.x);
            const float k1 = uv * (1.0f - c);
            wv.axis[kk] = make_float4(fmaf(cx, s, fmaf(v.x, c, k1 * ux)), fmaf(cy, s, fmaf(v.y, c, k1 * uy)),
                                      fmaf(cz, s, fmaf(v.z, c, k1 * uz)), 0.0f);
        }
    }
    __syncwarp();
    return t;
}

// ------------------------------------------------------------------ one ligand, one CTA
__device__ void dock_ligand_cta(const DockArgs &A, int l, char *sm) {
    const Layout &Ly = A.ly;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, W = blockDim.x >> 5;
    if (A.out.status[l] != LG_OK) return;  // rejected by the preparation kernel (uniform)
    const CtaView cv = cta_view(sm, Ly);
    const WarpView wv = warp_view(sm, Ly, warp);
    const BatchDev &B = A.batch;
    const PocketDev &Pk = A.pocket;
    const int a0 = B.atom_off[l], N = B.atom_off[l + 1] - a0;
    const int r0 = B.rot_off[l], R = B.rot_off[l + 1] - r0;
    const int S = A.S, P = A.P;

    // stage the ligand: centroid-relative coordinates in grid units (FP64
    // difference), topology, per-atom weights, bond vectors
    {
        const double cx = A.scr.centroid[3 * l], cy = A.scr.centroid[3 * l + 1], cz = A.scr.centroid[3 * l + 2];
        const double ih = (double)Pk.inv_h;
        for (int i = tid; i < N; i += blockDim.x) {
            cv.d0x[i] = (float)(((double)B.x[a0 + i] - cx) * ih);
            cv.d0y[i] = (float)(((double)B.y[a0 + i] - cy) * ih);
            cv.d0z[i] = (float)(((double)B.z[a0 + i] - cz) * ih);
            cv.par[i] = B.parent[a0 + i];
            cv.wq[i] = make_float2(Pk.type_w[B.type[a0 + i]], B.q[a0 + i]);
        }
        for (int k = tid; k < R; k += blockDim.x) {
            const int b = B.rot_child[r0 + k], p = B.parent[a0 + b];
            cv.rch[k] = b;
            cv.rend[k] = A.scr.rot_end[(size_t)l * A.rmax_lim + k];
            cv.dv[k] = make_float4((B.x[a0 + b] - B.x[a0 + p]) * Pk.inv_h, (B.y[a0 + b] - B.y[a0 + p]) * Pk.inv_h,
                                   (B.z[a0 + b] - B.z[a0 + p]) * Pk.inv_h, 0.0f);
        }
    }
    __syncthreads();

    // per-lane torsion steps: lane t owns step t, and step 32 + (t & 3) in the tail
    const float cl = c_cos[lane], sl = c_sin[lane];
    const float ct = c_cos[32 + (lane & 3)], st = c_sin[32 + (lane & 3)];
    const uint64_t uid = B.uid[l];
    const uint2 key = make_uint2(A.seed_lo, A.seed_hi);
    const GridK Go = grid_k(Pk, Pk.cell_o), Gve = grid_k(Pk, Pk.cell_ve);
    const int PR = P * R;

    double bestE = INFINITY;
    int bestR = -1;
    for (int r = warp; r < S; r += W) {
        // 1. restart pose
        const uint4 x4 = philox4x32_10(make_uint4((uint32_t)uid, (uint32_t)(uid >> 32), (uint32_t)r, 0u), key);
        const float u0 = (float)(x4.x >> 8) * 5.9604644775390625e-08f;  // 2^-24
        const float u1 = (float)(x4.y >> 8) * 5.9604644775390625e-08f;
        const float u2 = (float)(x4.z >> 8) * 5.9604644775390625e-08f;
        const float s1 = sqrtf(1.0f - u0), s2 = sqrtf(u0);
        float sn1, cs1, sn2, cs2;
        sincospif(2.0f * u1, &sn1, &cs1);
        sincospif(2.0f * u2, &sn2, &cs2);
        const float qx = s1 * sn1, qy = s1 * cs1, qz = s2 * sn2, qw = s2 * cs2;
        const float R00 = 1.0f - 2.0f * (qy * qy + qz * qz), R01 = 2.0f * (qx * qy - qw * qz), R02 = 2.0f * (qx * qz + qw * qy);
        const float R10 = 2.0f * (qx * qy + qw * qz), R11 = 1.0f - 2.0f * (qx * qx + qz * qz), R12 = 2.0f * (qy * qz - qw * qx);
        const float R20 = 2.0f * (qx * qz - qw * qy), R21 = 2.0f * (qy * qz + qw * qx), R22 = 1.0f - 2.0f * (qx * qx + qy * qy);
        const uint32_t ppi = (uint32_t)(((uint64_t)(x4.w >> 8) * (uint64_t)Pk.n_pp) >> 24);
        const float4 pp = __ldg(Pk.pp + ppi);
        for (int i = lane; i < N; i += 32) {
            const float vx = cv.d0x[i], vy = cv.d0y[i], vz = cv.d0z[i];
            wv.Xx[i] = fmaf(R00, vx, fmaf(R01, vy, fmaf(R02, vz, pp.x)));
            wv.Xy[i] = fmaf(R10, vx, fmaf(R11, vy, fmaf(R12, vz, pp.y)));
            wv.Xz[i] = fmaf(R20, vx, fmaf(R21, vy, fmaf(R22, vz, pp.z)));
        }
        for (int k = lane; k < R; k += 32) {
            const float4 v = cv.dv[k];
            wv.axis[k] = make_float4(fmaf(R00, v.x, fmaf(R01, v.y, R02 * v.z)), fmaf(R10, v.x, fmaf(R11, v.y, R12 * v.z)),
                                     fmaf(R20, v.x, fmaf(R21, v.y, R22 * v.z)), 0.0f);
        }
        __syncwarp();
        // 2. greedy torsion sweep
        for (int ps = 0; ps < P; ++ps)
            for (int k = 0; k < R; ++k) {
                const int t = sweep_bond(A, Go, cv, wv, N, R, k, lane, cl, sl, ct, st);
                if (lane == 0) wv.tcur[ps * R + k] = (uint8_t)t;
            }
        __syncwarp();
        // 3. pose score: FP32 per-atom terms, FP64 sum
        double E = 0.0;
        for (int i = lane; i < N; i += 32) {
            const float2 wq = cv.wq[i];
            E += (double)atom_energy(Pk, Gve, wv.Xx[i], wv.Xy[i], wv.Xz[i], wq.x, wq.y);
        }
        E = warp_sum_d(E);
        if (A.out.restart_score && lane == 0) A.out.restart_score[(size_t)l * S + r] = E;
        if (A.out.restart_tors)
            for (int t = lane; t < PR; t += 32) A.out.restart_tors[(size_t)S * P * r0 + (size_t)r * PR + t] = wv.tcur[t];
        // 4. best restart of this warp (restarts visited in ascending order)
        if (E < bestE) {
            bestE = E;
            bestR = r;
            for (int t = lane; t < PR; t += 32) wv.tbest[t] = wv.tcur[t];
            if (Ly.want_pose)
                for (int i = lane; i < N; i += 32) {
                    wv.Bx[i] = wv.Xx[i];
                    wv.By[i] = wv.Xy[i];
                    wv.Bz[i] = wv.Xz[i];
                }
        }
        __syncwarp();
    }
    if (lane == 0) {
        cv.wE[warp] = bestE;
        cv.wR[warp] = bestR;
    }
    __syncthreads();
    // best restart over warps: lowest E, then lowest restart
    int bw = -1;
    double be = INFINITY;
    int br = 0x7fffffff;
    for (int w = 0; w < W; ++w) {
        const int rr = cv.wR[w];
        if (rr < 0) continue;
        const double ee = cv.wE[w];
        if (bw < 0 || ee < be || (ee == be && rr < br)) {
            bw = w;
            be = ee;
            br = rr;
        }
    }
    if (bw < 0) {  // every restart produced a non-finite score
        if (tid == 0) {
            A.out.score[l] = __longlong_as_double(0x7ff8000000000000ll);
            A.out.best_restart[l] = -1;
            A.out.status[l] = LG_EINVAL;
        }
    } else {
        const WarpView bv = warp_view(sm, Ly, bw);
        if (tid == 0) {
            A.out.score[l] = be;
            A.out.best_restart[l] = br;
        }
        if (A.out.tors_idx)
            for (int t = tid; t < PR; t += blockDim.x) A.out.tors_idx[(size_t)P * r0 + t] = bv.tbest[t];
        if (A.out.pose && Ly.want_pose) {
            const float3 c = Pk.center;
            const float h = Pk.h;
            for (int i = tid; i < N; i += blockDim.x) {
                float *o = A.out.pose + 3 * (size_t)(a0 + i);
                o[0] = fmaf(bv.Bx[i], h, c.x);
                o[1] = fmaf(bv.By[i], h, c.y);
                o[2] = fmaf(bv.Bz[i], h, c.z);
            }
        }
    }
    __syncthreads();
}

// ------------------------------------------------------------------ kernels
__global__ void __launch_bounds__(1024) k_dock_plain(const __grid_constant__ DockArgs A, int l) {
    extern __shared__ __align__(16) char sm[];
    dock_ligand_cta(A, l, sm);
}

// Persistent: CTAs pull ligands from a device counter in cost order.
__global__ void __launch_bounds__(1024) k_dock_batched(const __grid_constant__ DockArgs A) {
    extern __shared__ __align__(16) char sm[];
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(A.work_counter, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= A.batch.L) break;
        const int l = A.order ? A.order[item] : item;
        dock_ligand_cta(A, l, sm);
    }
}

// Preparation, one thread per ligand: validates the ligand (sizes within the
// limits, parent[0] = -1, parent[i] < i, contiguous subtrees -- subtree size
// equals end - start --, types, finite coordinates, torsional children strictly
// ascending in [1, N-1]), writes the end of every torsional child's subtree,
// the centroid (FP64) and the ligand's status; with `sort` it also files the
// ligand into a log-scale cost bucket (4 per octave) of
//   cost ~ restarts * (passes * 36 * sum of moving atoms + 8 * atoms + 64).
__global__ void k_prep(const __grid_constant__ DockArgs A, int sort) {
    __shared__ int sh[kSortBuckets];
    if (sort)
        for (int t = threadIdx.x; t < kSortBuckets; t += blockDim.x) sh[t] = 0;
    __syncthreads();
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l < A.batch.L) {
        const BatchDev &B = A.batch;
        const int a0 = B.atom_off[l], N = B.atom_off[l + 1] - a0;
        const int r0 = B.rot_off[l], R = B.rot_off[l + 1] - r0;
        bool ok = N >= 1 && N <= A.nmax_lim && R >= 0 && R <= A.rmax_lim;
        long msum = 0;
        if (ok) {
            int endv[LG_MAX_ATOMS], size[LG_MAX_ATOMS];
            ok = B.parent[a0] == -1;
            double sx = 0.0, sy = 0.0, sz = 0.0;
            for (int i = 0; i < N && ok; i++) {
                endv[i] = i + 1;
                size[i] = 1;
                const float x = B.x[a0 + i], y = B.y[a0 + i], z = B.z[a0 + i];
                if (i > 0) {
                    const int p = B.parent[a0 + i];
                    ok = p >= 0 && p < i;
                }
                ok = ok && B.type[a0 + i] < LG_NUM_TYPES && isfinite(x) && isfinite(y) && isfinite(z);
                sx += x;
                sy += y;
                sz += z;
            }
            if (ok) {
                for (int i = N - 1; i >= 1; i--) {
                    const int p = B.parent[a0 + i];
                    endv[p] = max(endv[p], endv[i]);
                    size[p] += size[i];
                }
                for (int i = 0; i < N && ok; i++) ok = size[i] == endv[i] - i;
                int prev = 0;
                for (int k = 0; k < R && ok; k++) {
                    const int b = B.rot_child[r0 + k];
                    ok = b >= 1 && b < N && b > prev;
                    if (ok) {
                        A.scr.rot_end[(size_t)l * A.rmax_lim + k] = (int16_t)endv[b];
                        msum += endv[b] - b - 1;
                        prev = b;
                    }
                }
            }
            if (ok) {
                A.scr.centroid[3 * l] = sx / N;
                A.scr.centroid[3 * l + 1] = sy / N;
                A.scr.centroid[3 * l + 2] = sz / N;
            }
        }
        A.out.status[l] = ok ? LG_OK : LG_EINVAL;
        if (!ok) {
            A.out.score[l] = __longlong_as_double(0x7ff8000000000000ll);
            A.out.best_restart[l] = -1;
        }
        if (sort) {
            const double cost = ok ? (double)A.S * ((double)A.P * 36.0 * (double)msum + 8.0 * N + 64.0) : 1.0;
            int key = (int)(4.0 * log2(cost));
            key = max(0, min(kSortBuckets - 1, key));
            A.scr.keys[l] = key;
            atomicAdd(&sh[key], 1);
        }
    }
    __syncthreads();
    if (sort)
        for (int t = threadIdx.x; t < kSortBuckets; t += blockDim.x)
            if (sh[t]) atomicAdd(&A.scr.hist[t], sh[t]);
}

// Exclusive offsets of the buckets in descending key order (one warp).
__global__ void k_sort_scan(int32_t *hist) {
    const int lane = threadIdx.x;
    constexpr int per = kSortBuckets / 32;
    int v[per];
    int tot = 0;
#pragma unroll
    for (int j = 0; j < per; j++) {
        v[j] = hist[kSortBuckets - 1 - (lane * per + j)];
        tot += v[j];
    }
    int incl = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(LG_FULL, incl, o);
        if (lane >= o) incl += y;
    }
    int run = incl - tot;
#pragma unroll
    for (int j = 0; j < per; j++) {
        hist[kSortBuckets - 1 - (lane * per + j)] = run;
        run += v[j];
    }
}

__global__ void k_sort_scatter(int L, const int32_t *keys, int32_t *hist, int32_t *order) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l < L) order[atomicAdd(&hist[keys[l]], 1)] = l;
}

__global__ void k_score_poses(const __grid_constant__ PocketDev P, int L, const int32_t *atom_off, const float *xyz,
                              const float *q, const uint8_t *type, double *E) {
    const int lane = threadIdx.x & 31;
    const int l = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (l >= L) return;
    const GridK G = grid_k(P, P.cell_ve);
    const int a0 = atom_off[l], N = atom_off[l + 1] - a0;
    double acc = 0.0;
    for (int i = lane; i < N; i += 32) {
        const int t = type[a0 + i];
        const float w = t < LG_NUM_TYPES ? P.type_w[t] : 0.0f;
        const float *x = xyz + 3 * (size_t)(a0 + i);
        acc += (double)atom_energy(P, G, (x[0] - P.center.x) * P.inv_h, (x[1] - P.center.y) * P.inv_h,
                                   (x[2] - P.center.z) * P.inv_h, w, q[a0 + i]);
    }
    acc = warp_sum_d(acc);
    if (lane == 0) E[l] = acc;
}

__global__ void k_diag_philox(int n, const uint32_t *ctr, const uint32_t *key, uint32_t *out, int use_curand) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
    const uint2 k = make_uint2(key[2 * i], key[2 * i + 1]);
    const uint4 o = use_curand ? curand_Philox4x32_10(c, k) : philox4x32_10(c, k);
    out[4 * i] = o.x;
    out[4 * i + 1] = o.y;
    out[4 * i + 2] = o.z;
    out[4 * i + 3] = o.w;
}

// ------------------------------------------------------------------ host side
static size_t al256(size_t v) { return (v + 255) & ~(size_t)255; }

size_t scratch_bytes(int L, int rmax) {
    return al256(4 * (kSortBuckets + 1)) + 2 * al256(4 * (size_t)L) + al256(24 * (size_t)L) +
           al256(2 * (size_t)L * (rmax > 0 ? rmax : 1));
}

Scratch carve_scratch(void *base, int L, int rmax) {
    (void)rmax;
    char *p = (char *)base;
    Scratch s;
    s.hist = (int32_t *)p;
    p += al256(4 * (kSortBuckets + 1));
    s.keys = (int32_t *)p;
    p += al256(4 * (size_t)L);
    s.order = (int32_t *)p;
    p += al256(4 * (size_t)L);
    s.centroid = (double *)p;
    p += al256(24 * (size_t)L);
    s.rot_end = (int16_t *)p;
    return s;
}

cudaError_t dock_kernel_attributes(int W, int smem, int *ctas_per_sm) {
    cudaError_t e = cudaFuncSetAttribute(k_dock_batched, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, k_dock_batched, 32 * W, smem);
}

cudaError_t plain_kernel_attributes(int smem) {
    return cudaFuncSetAttribute(k_dock_plain, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

cudaError_t launch_prep(const DockArgs &a, bool sort, cudaStream_t s, int *launches) {
    const int L = a.batch.L;
    const int blocks = (L + 255) / 256;
    k_prep<<<blocks, 256, 0, s>>>(a, sort ? 1 : 0);
    *launches += 1;
    if (sort) {
        k_sort_scan<<<1, 32, 0, s>>>(a.scr.hist);
        k_sort_scatter<<<blocks, 256, 0, s>>>(L, a.scr.keys, a.scr.hist, a.scr.order);
        *launches += 2;
    }
    return cudaGetLastError();
}

cudaError_t launch_dock_plain(const DockArgs &a, int ligand, cudaStream_t s) {
    k_dock_plain<<<1, 32 * a.ly.W, a.ly.total, s>>>(a, ligand);
    return cudaGetLastError();
}

cudaError_t launch_dock_batched(const DockArgs &a, int grid, cudaStream_t s) {
    k_dock_batched<<<grid, 32 * a.ly.W, a.ly.total, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_score_poses(const PocketDev &p, int L, const int32_t *atom_off, const float *xyz,
                               const float *q, const uint8_t *type, double *E, cudaStream_t s) {
    const int threads = 256, per = threads / 32;
    k_score_poses<<<(L + per - 1) / per, threads, 0, s>>>(p, L, atom_off, xyz, q, type, E);
    return cudaGetLastError();
}

cudaError_t launch_diag_philox(int n, const uint32_t *ctr, const uint32_t *key, uint32_t *out, int use_curand,
                               cudaStream_t s) {
    k_diag_philox<<<(n + 255) / 256, 256, 0, s>>>(n, ctr, key, out, use_curand);
    return cudaGetLastError();
}

}  // namespace lg
