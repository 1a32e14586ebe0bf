// Docking kernels for sm_103a (GB300).
//
// The dock-and-score step of the paper (Sec. 3.1) on the GPU: one CTA docks
// one ligand, its warps share the ligand's topology in shared memory and each
// warp runs one restart at a time (restarts are tiled over the CTA's warps).
// Inside a warp the 36 torsion steps of a bond map onto lanes: lane t scores
// step t for every moving atom (steps 32..35 are spread over the warp in a
// short tail loop), so the per-step overlap sums need no cross-lane reduction
// and the choice of step is a 5-level shuffle argmax.  Moving atoms are
// processed in bundles of 32 (the paper's CUDA design also works in bundles
// of 32 atoms, Sec. 3.1): each lane builds the circle that one atom traces
// about the bond axis, x(theta) = p + e1 cos(theta) + e2 sin(theta), and every
// lane then evaluates its own step on that circle with two FMAs per
// coordinate.  Grids are read as one 32-byte cell of trilinear coefficients
// per lookup through the read-only path and stay resident in L2.
// The batched form is a persistent kernel that visits ligands in descending
// estimated cost (a counting sort on the device), the plain form launches one
// CTA per ligand with one warp per restart.
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
// Cell of an index-space point already clamped to [0, n-1]: floor by adding
// 1.5*2^23 with round-down (the integer part lands in the low mantissa bits),
// exact fractions, and the flat node index (k*n + j)*n + i.
__device__ __forceinline__ uint32_t cell_of(float gx, float gy, float gz, int n, float &fx, float &fy, float &fz) {
    const float M = 12582912.0f;  // 0x4B400000
    const float tx = __fadd_rd(gx, M), ty = __fadd_rd(gy, M), tz = __fadd_rd(gz, M);
    fx = gx - (tx - M);
    fy = gy - (ty - M);
    fz = gz - (tz - M);
    const uint32_t ix = __float_as_uint(tx) - 0x4B400000u;
    const uint32_t iy = __float_as_uint(ty) - 0x4B400000u;
    const uint32_t iz = __float_as_uint(tz) - 0x4B400000u;
    return (iz * (uint32_t)n + iy) * (uint32_t)n + ix;
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

// Overlap-field value at index-space point g (clamped to the box).
__device__ __forceinline__ float lookup_o(const float4 *__restrict__ cells, float gx, float gy, float gz, int n,
                                          float gmax) {
    gx = clampg(gx, gmax);
    gy = clampg(gy, gmax);
    gz = clampg(gz, gmax);
    float fx, fy, fz;
    const uint32_t c = cell_of(gx, gy, gz, n, fx, fy, fz);
    const float4 *p = cells + 2 * (size_t)c;
    const float4 lo = __ldg(p), hi = __ldg(p + 1);
    return cell_eval(lo, hi, fx, fy, fz);
}

// Per-atom energy term at a centred-frame position: type weight * vdW grid +
// charge * electrostatic grid at the clamped position, plus k_out times the
// distance outside the box.
__device__ __forceinline__ float atom_energy(const PocketDev &P, float x, float y, float z, float w, float q) {
    const float gx = fmaf(x, P.inv_h, P.c0), gy = fmaf(y, P.inv_h, P.c0), gz = fmaf(z, P.inv_h, P.c0);
    const float cx = clampg(gx, P.gmax), cy = clampg(gy, P.gmax), cz = clampg(gz, P.gmax);
    const float dx = gx - cx, dy = gy - cy, dz = gz - cz;
    const float out = P.h * sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
    float fx, fy, fz;
    const uint32_t c = cell_of(cx, cy, cz, P.n, fx, fy, fz);
    const float4 *p = P.cell_ve + 4 * (size_t)c;
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
    int *par, *rch, *rend, *wR, *scal;
    double *cen;
};

struct WarpView {
    float4 *bundle;  // 32 x 3 float4; also holds T (rotated moving atoms, SoA, 3 x 128 floats)
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
    v.scal = (int *)(sm + L.o_scal);
    v.cen = (double *)(sm + L.o_scal + 32);
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
// Sweeps bond k of the current pose held by this warp and applies the chosen
// step.  Returns the chosen step (0..35).
__device__ int sweep_bond(const DockArgs &A, const CtaView &cv, const WarpView &wv, int N, int R, int k, int lane,
                          float cl, float sl, float ct, float st) {
    const PocketDev &P = A.pocket;
    const int b = cv.rch[k], a = cv.par[b], e = cv.rend[k];
    const int m = e - b - 1;
    if (m <= 0) return 0;  // nothing moves: every step scores 0, step 0 wins

    const float xbx = wv.Xx[b], xby = wv.Xy[b], xbz = wv.Xz[b];
    const float4 ax = wv.axis[k];
    const float inv = rnorm3df(ax.x, ax.y, ax.z);
    const float ux = ax.x * inv, uy = ax.y * inv, uz = ax.z * inv;
    const float ih = P.inv_h, c0 = P.c0;

    float acc = 0.0f, acc_t = 0.0f;
    for (int base = b + 1; base < e; base += 32) {
        const int cnt = min(32, e - base);
        if (lane < cnt) {
            const int i = base + lane;
            const float dx = wv.Xx[i] - xbx, dy = wv.Xy[i] - xby, dz = wv.Xz[i] - xbz;
            const float w = fmaf(ux, dx, fmaf(uy, dy, uz * dz));
            const float px = fmaf(w, ux, xbx), py = fmaf(w, uy, xby), pz = fmaf(w, uz, xbz);
            const float e1x = fmaf(-w, ux, dx), e1y = fmaf(-w, uy, dy), e1z = fmaf(-w, uz, dz);
            const float e2x = fmaf(uy, dz, -uz * dy), e2y = fmaf(uz, dx, -ux * dz), e2z = fmaf(ux, dy, -uy * dx);
            wv.bundle[3 * lane + 0] = make_float4(fmaf(px, ih, c0), fmaf(py, ih, c0), fmaf(pz, ih, c0), e1x * ih);
            wv.bundle[3 * lane + 1] = make_float4(e1y * ih, e1z * ih, e2x * ih, e2y * ih);
            wv.bundle[3 * lane + 2] = make_float4(e2z * ih, 0.0f, 0.0f, 0.0f);
        }
        __syncwarp();
        // steps 0..31: lane t scores step t for every atom of the bundle
#pragma unroll 2
        for (int t = 0; t < cnt; ++t) {
            const float4 q0 = wv.bundle[3 * t], q1 = wv.bundle[3 * t + 1], q2 = wv.bundle[3 * t + 2];
            const float gx = fmaf(q1.z, sl, fmaf(q0.w, cl, q0.x));
            const float gy = fmaf(q1.w, sl, fmaf(q1.x, cl, q0.y));
            const float gz = fmaf(q2.x, sl, fmaf(q1.y, cl, q0.z));
            acc += lookup_o(P.cell_o, gx, gy, gz, P.n, P.gmax);
        }
        // steps 32..35: lane scores step 32 + (lane & 3) for atoms lane>>2, +8, ...
        for (int t = lane >> 2; t < cnt; t += 8) {
            const float4 q0 = wv.bundle[3 * t], q1 = wv.bundle[3 * t + 1], q2 = wv.bundle[3 * t + 2];
            const float gx = fmaf(q1.z, st, fmaf(q0.w, ct, q0.x));
            const float gy = fmaf(q1.w, st, fmaf(q1.x, ct, q0.y));
            const float gz = fmaf(q2.x, st, fmaf(q1.y, ct, q0.z));
            acc_t += lookup_o(P.cell_o, gx, gy, gz, P.n, P.gmax);
        }
        __syncwarp();
    }
    acc_t += __shfl_xor_sync(LG_FULL, acc_t, 4);
    acc_t += __shfl_xor_sync(LG_FULL, acc_t, 8);
    acc_t += __shfl_xor_sync(LG_FULL, acc_t, 16);

    // Highest-scoring admissible step, lowest step on ties.  Candidates are
    // tried in that order; step 0 (the current pose) is always admissible.
    float *Tx = (float *)wv.bundle;  // rotated moving atoms (SoA, up to 128 each)
    float *Ty = Tx + LG_MAX_ATOMS, *Tz = Ty + LG_MAX_ATOMS;
    const int nF = N - (e - b);  // atoms outside subtree(b)
    int removed = 0;             // bit 0: step lane, bit 1: step 32 + lane (lanes 0..3)
    int chosen = 0;
    for (;;) {
        float bs = (removed & 1) ? -INFINITY : acc;
        int ba = (removed & 1) ? 1024 : lane;
        if (lane < 4 && !(removed & 2) && acc_t > bs) {  // equal scores keep the lower step (lane < 32 + lane)
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
        if (t <= 0 || t >= LG_ANGLE_STEPS) break;  // step 0 is admissible by definition
        // rotated positions of the moving atoms for step t
        const float c = c_cos[t], s = c_sin[t];
        for (int i = b + 1 + lane; i < e; i += 32) {
            const float dx = wv.Xx[i] - xbx, dy = wv.Xy[i] - xby, dz = wv.Xz[i] - xbz;
            const float w = fmaf(ux, dx, fmaf(uy, dy, uz * dz));
            const float e1x = fmaf(-w, ux, dx), e1y = fmaf(-w, uy, dy), e1z = fmaf(-w, uz, dz);
            const float e2x = fmaf(uy, dz, -uz * dy), e2y = fmaf(uz, dx, -ux * dz), e2z = fmaf(ux, dy, -uy * dx);
            const int ii = i - b - 1;
            Tx[ii] = fmaf(e2x, s, fmaf(e1x, c, fmaf(w, ux, xbx)));
            Ty[ii] = fmaf(e2y, s, fmaf(e1y, c, fmaf(w, uy, xby)));
            Tz[ii] = fmaf(e2z, s, fmaf(e1z, c, fmaf(w, uz, xbz)));
        }
        __syncwarp();
        bool clash = false;
        for (int ii = 0; ii < m; ++ii) {
            const int i = b + 1 + ii;
            const float tx = Tx[ii], ty = Ty[ii], tz = Tz[ii];
            const bool child_of_b = (cv.par[i] == b);
            bool cl_l = false;
            for (int jj = lane; jj < nF; jj += 32) {
                const int j = jj < b ? jj : jj + (e - b);
                if (child_of_b && j == a) continue;  // two bonds apart through the bond itself
                const float dx = tx - wv.Xx[j], dy = ty - wv.Xy[j], dz = tz - wv.Xz[j];
                cl_l |= fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < A.dc2;
            }
            if (__any_sync(LG_FULL, cl_l)) {
                clash = true;
                break;
            }
        }
        if (!clash) {
            chosen = t;
            break;
        }
        if (t < 32) {
            if (lane == t) removed |= 1;
        } else if (lane == t - 32) {
            removed |= 2;
        }
        __syncwarp();
    }

    if (chosen != 0) {
        for (int i = b + 1 + lane; i < e; i += 32) {
            const int ii = i - b - 1;
            wv.Xx[i] = Tx[ii];
            wv.Xy[i] = Ty[ii];
            wv.Xz[i] = Tz[ii];
        }
        // bond axes further down the subtree turn with it
        const float c = c_cos[chosen], s = c_sin[chosen];
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
    }
    __syncwarp();
    return chosen;
}

// ------------------------------------------------------------------ one ligand, one CTA
__device__ void dock_ligand_cta(const DockArgs &A, int l, char *sm) {
    const Layout &Ly = A.ly;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, W = blockDim.x >> 5;
    const CtaView cv = cta_view(sm, Ly);
    const WarpView wv = warp_view(sm, Ly, warp);
    const BatchDev &B = A.batch;
    const int a0 = B.atom_off[l], N = B.atom_off[l + 1] - a0;
    const int r0 = B.rot_off[l], R = B.rot_off[l + 1] - r0;
    const int S = A.S, P = A.P;

    const bool size_ok = N >= 1 && N <= A.nmax_decl && N <= Ly.nmax && R >= 0 && R <= A.rmax_decl && R <= Ly.rmax;
    if (size_ok) {
        for (int i = tid; i < N; i += blockDim.x) {
            cv.d0x[i] = B.x[a0 + i];
            cv.d0y[i] = B.y[a0 + i];
            cv.d0z[i] = B.z[a0 + i];
            cv.par[i] = B.parent[a0 + i];
            const int t = B.type[a0 + i];
            cv.wq[i] = make_float2(t < LG_NUM_TYPES ? A.pocket.type_w[t] : 0.0f, B.q[a0 + i]);
        }
        for (int k = tid; k < R; k += blockDim.x) cv.rch[k] = B.rot_child[r0 + k];
    }
    __syncthreads();
    if (warp == 0) {
        // validation (lane 0, sequential over the atoms) and centroid (FP64)
        int ok = size_ok ? 1 : 0;
        if (ok && lane == 0) {
            // parent[i] < i, and every subtree contiguous: size(v) == end(v) - v
            int *endv = (int *)wv.Xx;  // scratch: warp 0's position buffers
            int *size = (int *)wv.Xy;
            if (cv.par[0] != -1) ok = 0;
            for (int i = 1; i < N && ok; i++)
                if (cv.par[i] < 0 || cv.par[i] >= i) ok = 0;
            for (int i = 0; i < N && ok; i++) {
                const int t = B.type[a0 + i];
                if (t >= LG_NUM_TYPES) ok = 0;
                if (!isfinite(cv.d0x[i]) || !isfinite(cv.d0y[i]) || !isfinite(cv.d0z[i])) ok = 0;
            }
            if (ok) {
                for (int i = 0; i < N; i++) { endv[i] = i + 1; size[i] = 1; }
                for (int i = N - 1; i >= 1; i--) {
                    const int p = cv.par[i];
                    endv[p] = max(endv[p], endv[i]);
                    size[p] += size[i];
                }
                for (int i = 0; i < N && ok; i++)
                    if (size[i] != endv[i] - i) ok = 0;
                for (int k = 0; k < R && ok; k++) {
                    const int b = cv.rch[k];
                    if (b < 1 || b >= N || (k > 0 && b <= cv.rch[k - 1])) ok = 0;
                    else cv.rend[k] = endv[b];
                }
            }
        }
        ok = __shfl_sync(LG_FULL, ok, 0);
        if (ok) {
            double sx = 0.0, sy = 0.0, sz = 0.0;
            for (int i = lane; i < N; i += 32) {
                sx += (double)cv.d0x[i];
                sy += (double)cv.d0y[i];
                sz += (double)cv.d0z[i];
            }
            sx = warp_sum_d(sx); sy = warp_sum_d(sy); sz = warp_sum_d(sz);
            if (lane == 0) {
                cv.cen[0] = sx / N;
                cv.cen[1] = sy / N;
                cv.cen[2] = sz / N;
            }
        }
        if (lane == 0) cv.scal[0] = ok;
    }
    __syncthreads();
    if (!cv.scal[0]) {
        if (tid == 0) {
            A.out.score[l] = __longlong_as_double(0x7ff8000000000000ll);
            A.out.best_restart[l] = -1;
            A.out.status[l] = LG_EINVAL;
        }
        __syncthreads();
        return;
    }
    // bond vectors from the input coordinates, then centroid-relative atoms
    for (int k = tid; k < R; k += blockDim.x) {
        const int b = cv.rch[k], a = cv.par[b];
        cv.dv[k] = make_float4(cv.d0x[b] - cv.d0x[a], cv.d0y[b] - cv.d0y[a], cv.d0z[b] - cv.d0z[a], 0.0f);
    }
    __syncthreads();
    {
        const double cx = cv.cen[0], cy = cv.cen[1], cz = cv.cen[2];
        for (int i = tid; i < N; i += blockDim.x) {
            cv.d0x[i] = (float)((double)cv.d0x[i] - cx);
            cv.d0y[i] = (float)((double)cv.d0y[i] - cy);
            cv.d0z[i] = (float)((double)cv.d0z[i] - cz);
        }
    }
    __syncthreads();

    // per-lane torsion steps: lane t owns step t, and step 32 + (t & 3) in the tail
    const float cl = c_cos[lane], sl = c_sin[lane];
    const float ct = c_cos[32 + (lane & 3)], st = c_sin[32 + (lane & 3)];
    const uint64_t uid = B.uid[l];
    const uint2 key = make_uint2(A.seed_lo, A.seed_hi);
    const PocketDev &Pk = A.pocket;
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
                const int t = sweep_bond(A, cv, wv, N, R, k, lane, cl, sl, ct, st);
                if (lane == 0) wv.tcur[ps * R + k] = (uint8_t)t;
            }
        __syncwarp();
        // 3. pose score: FP32 per-atom terms, FP64 sum
        double E = 0.0;
        for (int i = lane; i < N; i += 32) {
            const float2 wq = cv.wq[i];
            E += (double)atom_energy(Pk, wv.Xx[i], wv.Xy[i], wv.Xz[i], wq.x, wq.y);
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
            A.out.status[l] = LG_OK;
        }
        if (A.out.tors_idx)
            for (int t = tid; t < PR; t += blockDim.x) A.out.tors_idx[(size_t)P * r0 + t] = bv.tbest[t];
        if (A.out.pose && Ly.want_pose) {
            const float3 c = Pk.center;
            for (int i = tid; i < N; i += blockDim.x) {
                float *o = A.out.pose + 3 * (size_t)(a0 + i);
                o[0] = bv.Bx[i] + c.x;
                o[1] = bv.By[i] + c.y;
                o[2] = bv.Bz[i] + c.z;
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

// Cost estimate and bucket (log scale, 4 buckets per octave) of every ligand:
// cost ~ restarts * (passes * 36 * sum of moving atoms + atoms).
__global__ void k_sort_keys(const __grid_constant__ DockArgs A, int32_t *keys, int32_t *hist) {
    __shared__ int sh[kSortBuckets];
    for (int t = threadIdx.x; t < kSortBuckets; t += blockDim.x) sh[t] = 0;
    __syncthreads();
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l < A.batch.L) {
        const BatchDev &B = A.batch;
        const int a0 = B.atom_off[l], N = B.atom_off[l + 1] - a0;
        const int r0 = B.rot_off[l], R = B.rot_off[l + 1] - r0;
        double cost = 1.0;
        if (N >= 1 && N <= LG_MAX_ATOMS && R >= 0 && R <= LG_MAX_ROT) {
            int endv[LG_MAX_ATOMS];
            for (int i = 0; i < N; i++) endv[i] = i + 1;
            for (int i = N - 1; i >= 1; i--) {
                const int p = B.parent[a0 + i];
                if (p >= 0 && p < i) endv[p] = max(endv[p], endv[i]);
            }
            long msum = 0;
            for (int k = 0; k < R; k++) {
                const int b = B.rot_child[r0 + k];
                if (b >= 1 && b < N) msum += endv[b] - b - 1;
            }
            cost = (double)A.S * ((double)A.P * 36.0 * (double)msum + 8.0 * N + 64.0);
        }
        int key = (int)(4.0 * log2(cost));
        key = max(0, min(kSortBuckets - 1, key));
        keys[l] = key;
        atomicAdd(&sh[key], 1);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < kSortBuckets; t += blockDim.x)
        if (sh[t]) atomicAdd(&hist[t], sh[t]);
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
    const int a0 = atom_off[l], N = atom_off[l + 1] - a0;
    double acc = 0.0;
    for (int i = lane; i < N; i += 32) {
        const int t = type[a0 + i];
        const float w = t < LG_NUM_TYPES ? P.type_w[t] : 0.0f;
        const float *x = xyz + 3 * (size_t)(a0 + i);
        acc += (double)atom_energy(P, x[0] - P.center.x, x[1] - P.center.y, x[2] - P.center.z, w, q[a0 + i]);
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

// ------------------------------------------------------------------ launchers
cudaError_t dock_kernel_attributes(int W, int smem, int *ctas_per_sm) {
    cudaError_t e = cudaFuncSetAttribute(k_dock_batched, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, k_dock_batched, 32 * W, smem);
}

cudaError_t plain_kernel_attributes(int smem) {
    return cudaFuncSetAttribute(k_dock_plain, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

cudaError_t launch_dock_plain(const DockArgs &a, int ligand, cudaStream_t s) {
    k_dock_plain<<<1, 32 * a.ly.W, a.ly.total, s>>>(a, ligand);
    return cudaGetLastError();
}

cudaError_t launch_dock_batched(const DockArgs &a, int grid, cudaStream_t s) {
    k_dock_batched<<<grid, 32 * a.ly.W, a.ly.total, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_sort(const DockArgs &a, int32_t *keys, int32_t *hist, int32_t *order, cudaStream_t s,
                        int *launches) {
    const int L = a.batch.L;
    const int blocks = (L + 255) / 256;
    k_sort_keys<<<blocks, 256, 0, s>>>(a, keys, hist);
    k_sort_scan<<<1, 32, 0, s>>>(hist);
    k_sort_scatter<<<blocks, 256, 0, s>>>(L, keys, hist, order);
    *launches += 3;
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
