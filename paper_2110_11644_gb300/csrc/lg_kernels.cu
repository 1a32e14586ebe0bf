// Docking kernels for sm_103a (GB300): the dock-and-score step of the paper
// (Sec. 3.1) -- restart poses, greedy torsion sweep with clash check, grid
// scoring, best restart.  The per-step arithmetic is in lg_device.cuh.
//
// Two forms share it and produce bit-identical results (where a form has its
// own loop, it sums in the same order):
//
//  * k_dock_plain -- one CTA per ligand, one warp per restart, one launch per
//    ligand.  Lanes own torsion steps: lane t scores step t for every moving
//    atom (steps 32..35 by lanes 0..3), moving atoms are processed in bundles
//    of 32 (the paper's CUDA design works in bundles of 32 atoms, Sec. 3.1).
//
//  * k_dock_batched -- persistent, ligands in descending estimated cost.  One
//    CTA docks one ligand; each warp holds 8 restart slots at once with 4
//    lanes per restart, each lane owning 9 of the 36 steps, so the work that is
//    paid once per decision (circle set-up, argmax, moves) is shared by 8
//    restarts, the 9 steps of a lane (every 4th step) are straight-line code,
//    and the argmax needs 2 shuffles; a slot whose restart has finished takes
//    the warp's next restart at the next pass boundary.
//
// Every moving atom traces a circle about the bond axis,
//     x(theta) = p + e1 cos(theta) + e2 sin(theta),
// so a torsion step costs two FMAs per coordinate plus one 32-byte cell of
// trilinear coefficients of the overlap grid (L2-resident, read-only path).
// The clash test uses the same circles: for a moving atom i and a fixed atom j
//     |x_i(theta) - x_j|^2 = C + 2a cos(theta) + 2b sin(theta),
// whose minimum over the circle is C - 2 sqrt(a^2 + b^2).  Pairs that stay
// clear of d_clash at every step are dropped with one test; the others are
// evaluated step by step.  Fixed atoms outside the moving subtree's range of
// axial and radial coordinates about the bond (widened by d_clash) are never
// paired: a point's distance to a coaxial circle is at least the distance
// between the two in the (axial, radial) plane.
//
// Positions live in centred grid units (see lg_internal.h).
#include <curand_philox4x32_x.h>

#include <algorithm>

#include "lg_device.cuh"

namespace lg {

__constant__ float c_cos[LG_ANGLE_STEPS];

// decision_rank: bit 7 marks a decision skipped by an exact convergence stop
// (its low bits repeat the bond's previous rank)
constexpr uint8_t kRankSkipped = 0x80;
__constant__ float c_sin[LG_ANGLE_STEPS];

void set_angle_tables(const float *cosv, const float *sinv) {
    cudaMemcpyToSymbol(c_cos, cosv, sizeof(float) * LG_ANGLE_STEPS);
    cudaMemcpyToSymbol(c_sin, sinv, sizeof(float) * LG_ANGLE_STEPS);
}

// Bounds-check record of a debug build (see lg_device.cuh): waits for the
// stream, returns the failures and fills rec (site, index, bound, failures),
// then clears the record; 0 in other builds.
int checks_collect(cudaStream_t s, int rec[4]) {
#ifdef LG_CHECKS
    if (cudaStreamSynchronize(s) != cudaSuccess) return 0;
    cudaMemcpyFromSymbol(rec, lg_check_rec, sizeof(int) * 4);
    const int zero[4] = {0, 0, 0, 0};
    cudaMemcpyToSymbol(lg_check_rec, zero, sizeof(int) * 4);
    return rec[3];
#else
    (void)s;
    rec[0] = rec[1] = rec[2] = rec[3] = 0;
    return 0;
#endif
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(LG_FULL, v, o);
    return v;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(LG_FULL, v, o);
    return v;
}

// ------------------------------------------------------------------ the ligand of a CTA
struct CtaView {
    float4 *dv;
    double *wE;
    float *d0x, *d0y, *d0z;
    float2 *wq;
    int *par, *rch, *rend, *wR;
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

// Where a docked ligand comes from, with the constants that depend on its
// pocket's grid spacing: the launch's batch and constants for the batched
// kernels, the request's for the serving loop.
struct LigSrc {
    BatchDev batch;
    float dc2g, thr2g, rigid_shift_g;  // d_clash^2, cluster RMSD^2, rigid shift in grid units
};

__device__ __forceinline__ LigSrc launch_src(const DockArgs &A) {
    LigSrc q;
    q.batch = A.batch;
    q.dc2g = A.dc2g;
    q.thr2g = A.thr2g;
    q.rigid_shift_g = A.rigid_shift_g;
    return q;
}

// Stage ligand l: centroid-relative coordinates in grid units (FP64
// difference), parents, per-atom (type weight, charge), torsional children,
// subtree ends and input bond vectors in grid units.
__device__ __forceinline__ void stage_ligand(const DockArgs &A, const BatchDev &B, const PocketDev &Pk,
                                             const CtaView &cv, int l, int a0, int N, int r0, int R) {
    const size_t li = A.scr.per_cta ? (size_t)blockIdx.x : (size_t)l;  // the preparation's entry
    const double cx = A.scr.centroid[3 * li], cy = A.scr.centroid[3 * li + 1], cz = A.scr.centroid[3 * li + 2];
    const double ih = (double)Pk.inv_h;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        cv.d0x[i] = (float)(((double)B.x[a0 + i] - cx) * ih);
        cv.d0y[i] = (float)(((double)B.y[a0 + i] - cy) * ih);
        cv.d0z[i] = (float)(((double)B.z[a0 + i] - cz) * ih);
        cv.par[i] = B.parent[a0 + i];
        cv.wq[i] = make_float2(Pk.type_w[B.type[a0 + i]], B.q[a0 + i]);
    }
    for (int k = threadIdx.x; k < R; k += blockDim.x) {
        const int b = B.rot_child[r0 + k], p = B.parent[a0 + b];
        cv.rch[k] = b;
        cv.rend[k] = A.scr.rot_end[li * A.rmax_lim + k];
        cv.dv[k] = make_float4((B.x[a0 + b] - B.x[a0 + p]) * Pk.inv_h, (B.y[a0 + b] - B.y[a0 + p]) * Pk.inv_h,
                               (B.z[a0 + b] - B.z[a0 + p]) * Pk.inv_h, 0.0f);
    }
}

// Best restart over the CTA's warps (lowest E, then lowest restart) and the
// ligand's outputs.  Bx/By/Bz/tbest of the winning warp hold its best pose and
// decisions.  Returns after a CTA barrier.
template <typename BestOf>
__device__ __forceinline__ void finish_ligand(const DockArgs &A, const PocketDev &Pk, const OutDev &O, const CtaView &cv,
                                              int l, int a0, int N, int r0,
                                              int PR, BestOf best_of) {
    __syncthreads();
    const int W = blockDim.x >> 5, tid = threadIdx.x;
    int bw = -1, br = 0x7fffffff;
    double be = INFINITY;
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
            O.score[l] = __longlong_as_double(0x7ff8000000000000ll);
            O.best_restart[l] = -1;
            O.status[l] = LG_EINVAL;
        }
    } else {
        const float *Bx, *By, *Bz;
        const uint8_t *tb;
        best_of(bw, Bx, By, Bz, tb);
        if (tid == 0) {
            O.score[l] = be;
            O.best_restart[l] = br;
        }
        if (O.tors_idx)
            for (int t = tid; t < PR; t += blockDim.x) O.tors_idx[(size_t)A.P * r0 + t] = tb[t];
        if (O.pose && A.ly.want_pose) {
            const float3 c = Pk.center;
            const float h = Pk.h;
            for (int i = tid; i < N; i += blockDim.x) {
                float *o = O.pose + 3 * (size_t)(a0 + i);
                o[0] = fmaf(Bx[i], h, c.x);
                o[1] = fmaf(By[i], h, c.y);
                o[2] = fmaf(Bz[i], h, c.z);
            }
        }
    }
    __syncthreads();
}

// Keep restart r's final pose (centred grid units), score and decisions in
// the CTA's ranking slot.  X is the pose with a stride between atoms.
__device__ __forceinline__ size_t rk_pose_off(const DockArgs &A, int slot, int r) {
    return ((size_t)slot * A.S + r) * (size_t)A.ly.nmax * 3;
}

// The ranking step's geometric score G (the overlap grid summed over all
// atoms) and centroid of a restart's final pose, computed when the restart
// finishes: lane g of the 4 lanes that combine them sums atoms i = g (mod 4)
// in order (FP32); the partials are combined as (s0 + s1) + (s2 + s3), so
// both kernel forms produce the same numbers.
__device__ __forceinline__ float4 rank_geo_partial(const GridK &Go, float c0, const float *Xx, const float *Xy,
                                                   const float *Xz, int stride, int N, int g) {
    float s = 0.0f, cx = 0.0f, cy = 0.0f, cz = 0.0f;
    for (int i = g; i < N; i += 4) {
        const float x = Xx[i * stride], y = Xy[i * stride], z = Xz[i * stride];
        s += lookup_clamped(Go, x + c0, y + c0, z + c0);
        cx += x;
        cy += y;
        cz += z;
    }
    return make_float4(s, cx, cy, cz);
}

__device__ __forceinline__ float4 rank_geo_combine(float4 q) {  // over lanes 4k .. 4k+3
#pragma unroll
    for (int o = 1; o < 4; o <<= 1) {
        q.x += __shfl_xor_sync(LG_FULL, q.x, o);
        q.y += __shfl_xor_sync(LG_FULL, q.y, o);
        q.z += __shfl_xor_sync(LG_FULL, q.z, o);
        q.w += __shfl_xor_sync(LG_FULL, q.w, o);
    }
    return q;
}

// The ranking slot of a CTA (checked builds: within the slots the scratch
// holds at this launch's atom maximum).
__device__ __forceinline__ int rank_slot(const DockArgs &A, int slot) {
#ifdef LG_CHECKS
    const long long fit = (long long)(A.scr.rk_floats / ((size_t)A.S * A.ly.nmax * 3));
    return (int)LG_IDX(slot, fit < A.scr.rk_slots ? fit : A.scr.rk_slots, kChkRankSlot);
#else
    (void)A;
    return slot;
#endif
}

// Pose ranking (paper Sec. 3.1, steps 3-4) of ligand l from the restarts kept
// in the CTA's slot, and the ligand's outputs.  All threads of the CTA call it
// after a barrier; it reuses the warps' shared memory.
//   1. geometric score G_r = sum over atoms of the overlap grid (FP32 terms,
//      FP64 warp sum in a fixed order);
//   2. geometric order: higher G first, lower restart on ties;
//   3. greedy leader clustering in that order: a pose joins the first earlier
//      leader whose RMSD (no superposition) is at most the threshold;
//   4. ranking = leaders in order, then the other poses in order;
//   5. the lowest score among the first K ranked poses (lowest restart on ties).
// Step 3 first marks every pair within the threshold (a bit matrix), then walks
// the positions in order on one warp.  A pair is within the threshold when the
// FP32 sum of squared coordinate differences is at most thr^2 * N; pairs whose
// centroids are farther apart than the threshold (with a 1e-4 relative margin
// over the FP32 sum's rounding) cannot be, since the mean squared distance is
// at least the squared distance of the means, and skip the sum.
__device__ void rank_finish(const DockArgs &A, const PocketDev &Pk, const OutDev &O, float thr2g, int l, int slot, int a0,
                            int N, int r0, int PR, char *rbase) {
    const int S = A.S, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, W = blockDim.x >> 5;
    char *q = rbase;
    double *sG = (double *)q;
    q += lg_align16(8 * S);
    float *cen = (float *)q;    // [S][3], by restart
    q += lg_align16(24 * S);
    int *ord = (int *)q;        // restart at each geometric position
    q += lg_align16(4 * S);
    int *lpos = (int *)q;       // leader position of each geometric position
    q += lg_align16(4 * S);
    int *rk = (int *)q;         // ranked restarts
    q += lg_align16(4 * S);
    unsigned *bits = (unsigned *)q;
    q += lg_align16(4 * (rank_row_off(S) + 1));
    int *bestv = (int *)q;
    const float *pose0 = A.scr.rk_pose + rk_pose_off(A, slot, 0);
    const size_t pstride = (size_t)A.ly.nmax * 3;
    const bool cluster = thr2g > 0.0f;

    // 1. geometric scores and centroids, computed when each restart finished
    for (int r = tid; r < S; r += blockDim.x) {
        const size_t q = (size_t)slot * S + r;
        sG[r] = (double)A.scr.rk_G[q];
        cen[3 * r] = A.scr.rk_cen[3 * q] / (float)N;
        cen[3 * r + 1] = A.scr.rk_cen[3 * q + 1] / (float)N;
        cen[3 * r + 2] = A.scr.rk_cen[3 * q + 2] / (float)N;
    }
    __syncthreads();
    // 2. geometric order
    for (int r = tid; r < S; r += blockDim.x) {
        const double gr = sG[r];
        int c = 0;
        for (int o = 0; o < S; ++o) {
            const double go = sG[o];
            c += (go > gr) || (go == gr && o < r);
        }
        ord[c] = r;
    }
    __syncthreads();
    // 3a. pairs within the threshold: bit q of row p for positions q < p
    const float lim = thr2g * (float)N;
    if (cluster) {
        // the 1e-3 margin covers the FP32 rounding of the centroids (at most
        // ~1e-4 of the squared threshold for 100 atoms in the box)
        const float cut = thr2g * (1.0f + 1e-3f);
        for (int p = warp; p < S; p += W) {
            const int rp = ord[p];
            const float *x = pose0 + pstride * rp;
            const float px = cen[3 * rp], py = cen[3 * rp + 1], pz = cen[3 * rp + 2];
            for (int w = 0; 32 * w < p; ++w) {
                // pairs of this word that pass the centroid bound, then each
                // pair's sum of squared displacements by the whole warp
                // (coalesced: lane i takes coordinates i, i + 32, ...; FP32
                // lane sums combined in a fixed tree)
                const int qq = 32 * w + lane;
                bool cand = false;
                if (qq < p) {
                    const int rq = ord[qq];
                    const float dx = cen[3 * rq] - px, dy = cen[3 * rq + 1] - py, dz = cen[3 * rq + 2] - pz;
                    cand = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) <= cut;
                }
                unsigned todo = __ballot_sync(LG_FULL, cand), word = 0u;
                while (todo) {
                    const int bq = __ffs(todo) - 1;
                    todo &= todo - 1u;
                    const float *y = pose0 + pstride * ord[32 * w + bq];
                    float ss = 0.0f;
                    for (int i = lane; i < 3 * N; i += 32) {
                        const float d = x[i] - y[i];
                        ss = fmaf(d, d, ss);
                    }
                    if (warp_sum_f(ss) <= lim) word |= 1u << bq;
                }
                if (lane == 0) bits[rank_row_off(p) + w] = word;
            }
        }
    }
    __syncthreads();
    if (warp == 0) {
        // 3b. leaders in geometric order; lane w keeps word w of the leader set
        unsigned lead = 0;
        for (int p = 0; p < S; ++p) {
            const int nw = (p + 31) >> 5;
            const unsigned cand = (cluster && lane < nw) ? (bits[rank_row_off(p) + lane] & lead) : 0u;
            const unsigned any = __ballot_sync(LG_FULL, cand != 0u);
            if (any) {
                const int fw = __ffs(any) - 1;
                const unsigned c = __shfl_sync(LG_FULL, cand, fw);
                if (lane == 0) lpos[p] = 32 * fw + __ffs(c) - 1;
            } else {
                if (lane == (p >> 5)) lead |= 1u << (p & 31);
                if (lane == 0) lpos[p] = p;
            }
        }
        __syncwarp();
        // 4. ranking: leaders, then the others, each in geometric order
        int n = 0;
        for (int pass = 0; pass < 2; ++pass)
            for (int b0 = 0; b0 < S; b0 += 32) {
                const int p = b0 + lane;
                const bool take = p < S && ((lpos[p] == p) == (pass == 0));
                const unsigned bal = __ballot_sync(LG_FULL, take);
                if (take) rk[n + __popc(bal & ((1u << lane) - 1u))] = ord[p];
                n += __popc(bal);
            }
        __syncwarp();
        // 5. rescore the first K
        const int K = (A.rescore_top <= 0 || A.rescore_top > S) ? S : A.rescore_top;
        double be = INFINITY;
        int br = 0x7fffffff;
        for (int p = lane; p < K; p += 32) {
            const int r = rk[p];
            const double e = A.scr.rk_E[(size_t)slot * S + r];
            if (e < be || (e == be && r < br)) {
                be = e;
                br = r;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double oe = __shfl_xor_sync(LG_FULL, be, o);
            const int orr = __shfl_xor_sync(LG_FULL, br, o);
            if (oe < be || (oe == be && orr < br)) {
                be = oe;
                br = orr;
            }
        }
        if (lane == 0) {
            const bool ok = br != 0x7fffffff && isfinite(be);
            bestv[0] = ok ? br : -1;
            O.score[l] = ok ? be : __longlong_as_double(0x7ff8000000000000ll);
            O.best_restart[l] = ok ? br : -1;
            if (!ok) O.status[l] = LG_EINVAL;
        }
    }
    __syncthreads();
    const int br = bestv[0];
    if (br >= 0) {
        if (O.tors_idx)
            for (int t = tid; t < PR; t += blockDim.x)
                O.tors_idx[(size_t)A.P * r0 + t] = A.scr.rk_tors[((size_t)slot * S + br) * A.P * A.ly.rmax + t];
        if (O.pose) {
            const float *x = pose0 + pstride * br;
            const float3 c = Pk.center;
            for (int i = tid; i < N; i += blockDim.x) {
                float *o = O.pose + 3 * (size_t)(a0 + i);
                o[0] = fmaf(x[3 * i], Pk.h, c.x);
                o[1] = fmaf(x[3 * i + 1], Pk.h, c.y);
                o[2] = fmaf(x[3 * i + 2], Pk.h, c.z);
            }
        }
    }
    for (int p = tid; p < S; p += blockDim.x) {
        if (O.rank) O.rank[(size_t)l * S + p] = rk[p];
        if (O.leader) O.leader[(size_t)l * S + ord[p]] = ord[lpos[p]];
        if (O.restart_geo) O.restart_geo[(size_t)l * S + ord[p]] = sG[ord[p]];
    }
    __syncthreads();
}

// ================================================================== plain form
struct WarpView {
    float4 *bundle;  // 32 atoms x 4 float4 (see sweep_bond_plain); also per-atom energy terms
    float4 *axis;
    float *Xx, *Xy, *Xz;
    float *Bx, *By, *Bz;
    uint8_t *tcur, *tbest;
};

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

// One torsion decision of the warp's restart.  Bundle entry of a moving atom:
//   q0 = (P.x, P.y, P.z, e1.x), q1 = (e1.y, e1.z, e2.x, e2.y),
//   q2 = (e2.z, r2, inside, 0), q3 = (p.x, p.y, p.z, 0).
__device__ int sweep_bond_plain(const DockArgs &A, const GridK &G, const CtaView &cv, const WarpView &wv, int N,
                                int R, int k, int lane, float cl, float sl, float ct, float st, int &jr) {
    const int b = cv.rch[k], a = cv.par[b], e = cv.rend[k];
    const int m = e - b - 1;
    jr = 1;
    if (m <= 0) return 0;  // nothing moves: every step scores 0, step 0 wins

    const float xbx = wv.Xx[b], xby = wv.Xy[b], xbz = wv.Xz[b];
    const float3 u = unit_axis(wv.axis[k]);
    const float dc2 = A.dc2g;
    const int nF = N - (e - b);  // atoms outside subtree(b): [0, b) and [e, N)

    float acc = 0.0f, acc_t = 0.0f;
    bool clash_lo = false, clash_hi = false;
    for (int base = b + 1; base < e; base += 32) {
        const int cnt = min(32, e - base);
        if (lane < cnt) {
            const int i = base + lane;
            const Circle C = make_circle(wv.Xx[i], wv.Xy[i], wv.Xz[i], xbx, xby, xbz, u, 0.5f * G.gmax, G.gmax);
            float4 *q = wv.bundle + 4 * lane;
            q[0] = make_float4(C.Px, C.Py, C.Pz, C.e1x);
            q[1] = make_float4(C.e1y, C.e1z, C.e2x, C.e2y);
            q[2] = make_float4(C.e2z, C.r2, C.inside ? 1.0f : 0.0f, 0.0f);
            q[3] = make_float4(C.px, C.py, C.pz, 0.0f);
        }
        __syncwarp();
        for (int t = 0; t < cnt; ++t) {
            const float4 q0 = wv.bundle[4 * t], q1 = wv.bundle[4 * t + 1], q2 = wv.bundle[4 * t + 2];
            const float3 g = circle_index(q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w, q2.x, cl, sl);
            acc += (q2.z != 0.0f) ? lookup_in(G, g.x, g.y, g.z) : lookup_clamped(G, g.x, g.y, g.z);
        }
        if (lane < 4)  // steps 32..35, atoms in order
            for (int t = 0; t < cnt; ++t) {
                const float4 q0 = wv.bundle[4 * t], q1 = wv.bundle[4 * t + 1], q2 = wv.bundle[4 * t + 2];
                const float3 g = circle_index(q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w, q2.x, ct, st);
                acc_t += lookup_clamped(G, g.x, g.y, g.z);
            }
        // clash pairs (bundle atom ti, fixed atom jj), flattened over the warp
        const int npairs = cnt * nF;
        int ti = lane / nF, jj = lane - (lane / nF) * nF;
        for (int pb = 0; pb < npairs; pb += 32) {
            PairC q;
            q.near = false;
            q.C = q.A2 = q.B2 = 0.0f;
            if (pb + lane < npairs) {
                const int j = jj < b ? jj : jj + (e - b);
                if (!(j == a && cv.par[base + ti] == b)) {  // two bonds apart through the bond itself
                    const float4 *qq = wv.bundle + 4 * ti;
                    const float4 q0 = qq[0], q1 = qq[1], q2 = qq[2], q3 = qq[3];
                    q = pair_coeffs(q3.x, q3.y, q3.z, q0.w, q1.x, q1.y, q1.z, q1.w, q2.x, q2.y, wv.Xx[j], wv.Xy[j],
                                    wv.Xz[j], dc2);
                }
            }
            unsigned msk = __ballot_sync(LG_FULL, q.near);
            while (msk) {
                const int src = __ffs(msk) - 1;
                msk &= msk - 1;
                const float Cs = __shfl_sync(LG_FULL, q.C, src);
                const float As = __shfl_sync(LG_FULL, q.A2, src);
                const float Bs = __shfl_sync(LG_FULL, q.B2, src);
                clash_lo |= pair_clash(Cs, As, Bs, cl, sl, dc2);
                clash_hi |= pair_clash(Cs, As, Bs, ct, st, dc2);
            }
            jj += 32;
            while (jj >= nF) {
                jj -= nF;
                ++ti;
            }
        }
        __syncwarp();
    }
    if (lane == 0) clash_lo = false;  // step 0 (the current pose) is always admissible

    // highest-scoring admissible step, lowest step on ties
    float bs = clash_lo ? -INFINITY : acc;
    int ba = clash_lo ? 1024 : lane;
    if (lane < 4 && !clash_hi && acc_t > bs) {
        bs = acc_t;
        ba = 32 + lane;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float os = __shfl_xor_sync(LG_FULL, bs, o);
        const int oa = __shfl_xor_sync(LG_FULL, ba, o);
        if (better(os, oa, bs, ba)) {
            bs = os;
            ba = oa;
        }
    }
    const int t0 = __shfl_sync(LG_FULL, ba, 0);  // lane 0's copy keeps control flow warp-uniform
    const int t = (t0 > 0 && t0 < LG_ANGLE_STEPS) ? t0 : 0;
    if (A.out.decision_rank) {  // steps ranked before the chosen one, admissible or not
        const float bsu = __shfl_sync(LG_FULL, bs, 0);
        const unsigned lo = __ballot_sync(LG_FULL, acc > bsu || (acc == bsu && lane < t));
        const unsigned hi = __ballot_sync(LG_FULL, lane < 4 && (acc_t > bsu || (acc_t == bsu && 32 + lane < t)));
        jr = 1 + __popc(lo) + __popc(hi);
    }
    if (t == 0) return 0;

    const float c = c_cos[t], s = c_sin[t];
    for (int i = b + 1 + lane; i < e; i += 32) {
        const float3 x = rotate_point(wv.Xx[i], wv.Xy[i], wv.Xz[i], xbx, xby, xbz, u, c, s);
        wv.Xx[i] = x.x;
        wv.Xy[i] = x.y;
        wv.Xz[i] = x.z;
    }
    for (int kk = k + 1 + lane; kk < R; kk += 32)  // bond axes further down turn with it
        if (cv.rch[kk] < e) wv.axis[kk] = rotate_vec(wv.axis[kk], u, c, s);
    __syncwarp();
    return t;
}

// Rigid greedy moves of the warp's restart (plain form): lane c scores
// candidate c (same arithmetic and order as the restart-tiled form, so both
// forms choose and move identically).
__device__ __forceinline__ bool rigid_moves_plain(const DockArgs &A, const GridK &Go, const OutDev &O,
                                                  const WarpView &wv, int l, int r, int ps, int N, int R, int lane) {
    const float c0 = 0.5f * Go.gmax, dg = A.rigid_shift_g, ca = c_cos[1], sa = c_sin[1];
    bool moved = false;
    for (int j = 0; j < A.rigid_steps; ++j) {
        float sx = 0.0f, sy = 0.0f, sz = 0.0f;
        if (lane < 4)
            for (int i = lane; i < N; i += 4) {
                sx += wv.Xx[i];
                sy += wv.Xy[i];
                sz += wv.Xz[i];
            }
        sx += __shfl_xor_sync(LG_FULL, sx, 1);
        sy += __shfl_xor_sync(LG_FULL, sy, 1);
        sz += __shfl_xor_sync(LG_FULL, sz, 1);
        sx += __shfl_xor_sync(LG_FULL, sx, 2);
        sy += __shfl_xor_sync(LG_FULL, sy, 2);
        sz += __shfl_xor_sync(LG_FULL, sz, 2);
        sx = __shfl_sync(LG_FULL, sx, 0);
        sy = __shfl_sync(LG_FULL, sy, 0);
        sz = __shfl_sync(LG_FULL, sz, 0);
        const float cx = sx / (float)N, cy = sy / (float)N, cz = sz / (float)N;
        // lane c scores candidate c: FP32 sums s_g over atoms i = g (mod 4) in
        // order, combined as (s0 + s1) + (s2 + s3) (the batched form's order)
        float bG = -INFINITY;
        int bC = kRigidCandidates;
        if (lane < kRigidCandidates) {
            float s4[kLanesPerRestart];
#pragma unroll
            for (int g = 0; g < kLanesPerRestart; ++g) {
                s4[g] = 0.0f;
                for (int i = g; i < N; i += kLanesPerRestart) {
                    const float3 y = rigid_candidate(lane, wv.Xx[i], wv.Xy[i], wv.Xz[i], cx, cy, cz, dg, ca, sa);
                    s4[g] += lookup_clamped(Go, y.x + c0, y.y + c0, y.z + c0);
                }
            }
            bG = (s4[0] + s4[1]) + (s4[2] + s4[3]);
            bC = lane;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float oG = __shfl_xor_sync(LG_FULL, bG, o);
            const int oC = __shfl_xor_sync(LG_FULL, bC, o);
            if (oG > bG || (oG == bG && oC < bC)) {
                bG = oG;
                bC = oC;
            }
        }
        if (lane == 0 && O.restart_rigid)
            O.restart_rigid[(((size_t)l * A.S + r) * A.P + ps) * A.rigid_steps + j] = (uint8_t)bC;
        __syncwarp();
        moved = moved || bC != 0;
        if (bC != 0) {
            for (int i = lane; i < N; i += 32) {
                const float3 y = rigid_candidate(bC, wv.Xx[i], wv.Xy[i], wv.Xz[i], cx, cy, cz, dg, ca, sa);
                wv.Xx[i] = y.x;
                wv.Xy[i] = y.y;
                wv.Xz[i] = y.z;
            }
            for (int k = lane; k < R; k += 32) wv.axis[k] = rigid_candidate_vec(bC, wv.axis[k], ca, sa);
        }
        __syncwarp();
    }
    return moved;
}

__global__ void __launch_bounds__(1024) k_dock_plain(const __grid_constant__ DockArgs A, int l, int slot_arg) {
    extern __shared__ __align__(16) char sm[];
    if (A.out.status[l] != LG_OK) return;  // rejected by the preparation kernel
    const int slot = A.ranking ? rank_slot(A, slot_arg) : slot_arg;
    const Layout &Ly = A.ly;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
    const CtaView cv = cta_view(sm, Ly);
    const WarpView wv = warp_view(sm, Ly, warp);
    const BatchDev &B = A.batch;
    const PocketDev &Pk = A.pocket;
    const int a0 = B.atom_off[l], N = B.atom_off[l + 1] - a0;
    const int r0 = B.rot_off[l], R = B.rot_off[l + 1] - r0;
    const int S = A.S, P = A.P, PR = P * R;
    stage_ligand(A, B, Pk, cv, l, a0, N, r0, R);
    __syncthreads();

    const float cl = c_cos[lane], sl = c_sin[lane];
    const float ct = c_cos[32 + (lane & 3)], st = c_sin[32 + (lane & 3)];
    const uint64_t uid = B.uid[l];
    const uint2 key = make_uint2(A.seed_lo, A.seed_hi);
    const GridK Go = grid_k(Pk, Pk.cell_o), Gve = grid_k(Pk, Pk.cell_ve);
    float *eterm = (float *)wv.bundle;

    double bestE = INFINITY;
    int bestR = -1;
    for (int r = warp; r < S; r += W) {
        const Pose pose = restart_pose(uid, (uint32_t)r, key, Pk.n_pp);
        const float4 pp = __ldg(Pk.pp + pose.pp);
        for (int i = lane; i < N; i += 32) {
            const float3 x = rot_add(pose.R, cv.d0x[i], cv.d0y[i], cv.d0z[i], pp.x, pp.y, pp.z);
            wv.Xx[i] = x.x;
            wv.Xy[i] = x.y;
            wv.Xz[i] = x.z;
        }
        for (int k = lane; k < R; k += 32) {
            const float4 v = cv.dv[k];
            const float3 w = rot_vec(pose.R, v.x, v.y, v.z);
            wv.axis[k] = make_float4(w.x, w.y, w.z, 0.0f);
        }
        __syncwarp();
        // the same exact stops as the restart-tiled form, per restart: R
        // decisions in a row without a move (torsions only), or a pass without
        // a move (with rigid moves); the remaining decisions are step 0
        uint8_t *dr = A.out.decision_rank ? A.out.decision_rank + (size_t)S * P * r0 + (size_t)r * PR : nullptr;
        int zrun = 0;
        bool converged = false;
        for (int ps = 0; ps < P && !converged; ++ps) {
            bool moved = false;
            for (int k = 0; k < R; ++k) {
                int jr;
                const int t = sweep_bond_plain(A, Go, cv, wv, N, R, k, lane, cl, sl, ct, st, jr);
                if (lane == 0) {
                    wv.tcur[ps * R + k] = (uint8_t)t;
                    if (dr) dr[ps * R + k] = (uint8_t)jr;
                }
                moved = moved || t != 0;
                zrun = t != 0 ? 0 : zrun + 1;
                if (A.rigid_steps == 0 && zrun >= R) {
                    for (int q = ps * R + k + 1 + lane; q < P * R; q += 32) wv.tcur[q] = 0;
                    if (dr && lane == 0)  // skipped decisions repeat the bond's previous one, marked skipped
                        for (int q = ps * R + k + 1; q < P * R; ++q) dr[q] = dr[q - R] | kRankSkipped;
                    converged = true;
                    break;
                }
            }
            if (converged) break;
            if (A.rigid_steps > 0) moved = rigid_moves_plain(A, Go, A.out, wv, l, r, ps, N, R, lane) || moved;
            if (ps + 1 < P && !moved) {
                for (int q = (ps + 1) * R + lane; q < P * R; q += 32) wv.tcur[q] = 0;
                if (dr && lane == 0)
                    for (int q = (ps + 1) * R; q < P * R; ++q) dr[q] = dr[q - R] | kRankSkipped;
                if (A.rigid_steps > 0 && lane == 0 && A.out.restart_rigid)
                    for (int q = (ps + 1) * A.rigid_steps; q < P * A.rigid_steps; ++q)
                        A.out.restart_rigid[((size_t)l * S + r) * P * A.rigid_steps + q] = 0;
                break;
            }
        }
        __syncwarp();
        // pose score: FP32 per-atom terms; FP64 sums s_g over atoms i = g (mod 4)
        // in order, combined as (s0 + s1) + (s2 + s3)
        for (int i = lane; i < N; i += 32) {
            const float2 wq = cv.wq[i];
            eterm[i] = atom_energy(Pk, Gve, wv.Xx[i], wv.Xy[i], wv.Xz[i], wq.x, wq.y);
        }
        __syncwarp();
        double E = 0.0;
        if (lane < 4)
            for (int i = lane; i < N; i += 4) E += (double)eterm[i];
        E += __shfl_xor_sync(LG_FULL, E, 1);
        E += __shfl_xor_sync(LG_FULL, E, 2);
        E = __shfl_sync(LG_FULL, E, 0);
        if (A.out.restart_score && lane == 0) A.out.restart_score[(size_t)l * S + r] = E;
        if (A.out.restart_tors)
            for (int t = lane; t < PR; t += 32) A.out.restart_tors[(size_t)S * P * r0 + (size_t)r * PR + t] = wv.tcur[t];
        if (A.ranking) {  // keep the restart for the ranking step
            float *x = A.scr.rk_pose + rk_pose_off(A, slot, r);
            for (int i = lane; i < N; i += 32) {
                x[3 * i] = wv.Xx[i];
                x[3 * i + 1] = wv.Xy[i];
                x[3 * i + 2] = wv.Xz[i];
            }
            for (int t = lane; t < PR; t += 32) A.scr.rk_tors[((size_t)slot * S + r) * P * Ly.rmax + t] = wv.tcur[t];
            float4 gq = make_float4(0.0f, 0.0f, 0.0f, 0.0f);  // lanes 0..3 as the 4 lanes of a restart slot
            if (lane < 4) gq = rank_geo_partial(Go, Pk.c0, wv.Xx, wv.Xy, wv.Xz, 1, N, lane);
            gq = rank_geo_combine(gq);
            if (lane == 0) {
                const size_t q = (size_t)slot * S + r;
                A.scr.rk_E[q] = E;
                A.scr.rk_G[q] = gq.x;
                A.scr.rk_cen[3 * q] = gq.y;
                A.scr.rk_cen[3 * q + 1] = gq.z;
                A.scr.rk_cen[3 * q + 2] = gq.w;
            }
        }
        if (E < bestE) {  // restarts visited in ascending order: ties keep the lower one
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
    if (A.ranking) {
        __syncthreads();
        rank_finish(A, Pk, A.out, A.thr2g, l, slot, a0, N, r0, PR, sm + Ly.cta_bytes);
        return;
    }
    if (lane == 0) {
        cv.wE[warp] = bestE;
        cv.wR[warp] = bestR;
    }
    finish_ligand(A, Pk, A.out, cv, l, a0, N, r0, PR, [&](int w, const float *&Bx, const float *&By, const float *&Bz,
                                                         const uint8_t *&tb) {
        const WarpView bv = warp_view(sm, Ly, w);
        Bx = bv.Bx;
        By = bv.By;
        Bz = bv.Bz;
        tb = bv.tbest;
    });
}

// ================================================================== restart-tiled form
// Restart tile of a warp: LPR lanes per restart (2, 4, 8 or 16) and 32 / LPR
// restart slots; lane g of a restart owns the steps g, g + LPR, ...
// (ceil(36 / LPR) of them).  With 8 or 16 lanes the last round is ragged: its
// missing steps are evaluated at step 0's angle and never chosen.  Sums whose
// rounding reaches a result (pose score, rigid candidates and centroid, the
// ranking's geometric score) keep one order in every tile -- partial sums s_g
// over atoms i = g (mod 4) in order, combined as (s0 + s1) + (s2 + s3) -- and
// a step's score sums its moving atoms in order in one lane, so every tile
// gives the same bits.
template <int LPR>
struct Rt {
    static_assert(LPR == 2 || LPR == 4 || LPR == 8 || LPR == 16, "lanes per restart");
    static constexpr int slots = 32 / LPR;
    static constexpr int steps = (LG_ANGLE_STEPS + LPR - 1) / LPR;
    static constexpr bool ragged = steps * LPR != LG_ANGLE_STEPS;
    static constexpr int first_missing = LG_ANGLE_STEPS - LPR * (steps - 1);  // lanes g >= this lack the last step
    static constexpr unsigned gbits = (1u << LPR) - 1u;
    static constexpr int max_warps = LPR > 4 ? LPR : 4;  // warps per CTA the launch bounds allow
};

struct RtView {
    float4 *axis;          // [rmax][slots]
    float *Xx, *Xy, *Xz;   // [nmax][slots]
    float4 *pool;          // [kPoolCap] flagged clash pairs (C, A2, B2, restart slot)
    unsigned *mask;        // [32] clash bits of each lane's steps
    uint8_t *near;         // [slots][nstride] fixed atoms that can come within d_clash
    int nstride;
    float *Bx, *By, *Bz;   // [nmax] best pose of the warp
    uint8_t *tcur;         // [P*R][slots]
    uint8_t *tbest;        // [P*R]
};

template <int LPR>
__device__ __forceinline__ RtView rt_view(char *sm, const Layout &L, const LayoutRT &T, int w) {
    char *b = sm + L.cta_bytes + w * T.warp_bytes;
    RtView v;
    v.axis = (float4 *)(b + T.o_axis);
    v.Xx = (float *)(b + T.o_X);
    v.Xy = v.Xx + L.nmax * Rt<LPR>::slots;
    v.Xz = v.Xy + L.nmax * Rt<LPR>::slots;
    v.pool = (float4 *)(b + T.o_pool);
    v.mask = (unsigned *)(b + T.o_mask);
    v.near = (uint8_t *)(b + T.o_near);
    v.nstride = T.near_stride;
    v.Bx = (float *)(b + T.o_best);
    v.By = v.Bx + L.nmax;
    v.Bz = v.By + L.nmax;
    v.tcur = (uint8_t *)(b + T.o_tcur);
    v.tbest = (uint8_t *)(b + T.o_tbest);
    return v;
}

// K sums over atoms 0..N-1 in the tile-independent order: add(i, acc) adds
// atom i's K terms; s_g over i = g (mod 4) in order, combined as
// (s0 + s1) + (s2 + s3).  Lanes with on = false add nothing.  Every lane of
// the restart gets the sums.  All lanes of the warp call it.
template <int LPR, int K, typename T, typename F>
__device__ __forceinline__ void sum4(int g, int N, bool on, T (&out)[K], F &&add) {
    T a[K];
#pragma unroll
    for (int k = 0; k < K; ++k) a[k] = T(0);
    if constexpr (LPR == 2) {  // lane g holds s_g and s_(g+2)
        T b[K];
#pragma unroll
        for (int k = 0; k < K; ++k) b[k] = T(0);
        if (on) {
            for (int i = g; i < N; i += 4) add(i, a);
            for (int i = g + 2; i < N; i += 4) add(i, b);
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            a[k] += __shfl_xor_sync(LG_FULL, a[k], 1);
            b[k] += __shfl_xor_sync(LG_FULL, b[k], 1);
            out[k] = a[k] + b[k];
        }
    } else {  // lanes g < 4 hold s_g
        if (on && g < 4)
            for (int i = g; i < N; i += 4) add(i, a);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            a[k] += __shfl_xor_sync(LG_FULL, a[k], 1);
            a[k] += __shfl_xor_sync(LG_FULL, a[k], 2);
            if constexpr (LPR > 4) a[k] = __shfl_sync(LG_FULL, a[k], (int)(threadIdx.x & 31) & ~(LPR - 1));
            out[k] = a[k];
        }
    }
}

// Evaluate the pooled flagged pairs: in each round every restart group takes
// one entry (of any restart) and each of its lanes ORs the clash bits of its
// own steps into that restart's mask word for the same lane position.
template <int LPR>
__device__ __forceinline__ void flush_pool(const RtView &v, int rs, int g, int &pc, const float *cs, const float *sn,
                                           float dc2) {
    __syncwarp();
    for (int base = 0; base < pc; base += Rt<LPR>::slots) {
        const int e = base + rs;
        if (e < pc) {
            const float4 q = v.pool[e];
            unsigned bits = 0;
#pragma unroll
            for (int j = 0; j < Rt<LPR>::steps; ++j)
                bits |= (unsigned)pair_clash(q.x, q.y, q.z, cs[j], sn[j], dc2) << j;
            if (bits) atomicOr(&v.mask[LPR * __float_as_int(q.w) + g], bits);
        }
    }
    __syncwarp();
    pc = 0;
}

// One torsion decision for the warp's restart slots.  Lane = LPR*rs + g:
// restart slot rs, steps g, g+LPR, ... (cosines cs[], sines sn[]) -- the lanes
// of a restart score neighbouring steps in the same instruction.  Returns the
// step chosen for the lane's restart.
template <int LPR>
__device__ __forceinline__ int sweep_bond_rt(float dc2g, const GridK &G, const CtaView &cv, const RtView &v, int N, int R,
                                             int k, int rs, int g, bool valid, const float *cs, const float *sn,
                                             bool want_rank, int &jr) {
    using T = Rt<LPR>;
    constexpr int ST = T::slots;
    const int b = cv.rch[k], a = cv.par[b], e = cv.rend[k];
    const int m = e - b - 1;
    jr = 1;
    if (m <= 0) return 0;  // nothing moves: every step scores 0, step 0 wins

    const float xbx = v.Xx[b * ST + rs], xby = v.Xy[b * ST + rs], xbz = v.Xz[b * ST + rs];
    const float3 u = unit_axis(v.axis[k * ST + rs]);
    const float c0 = 0.5f * G.gmax, dc2 = dc2g;  // (n - 1) / 2, exact
    const int nF = N - (e - b);
    const int lane = LPR * rs + g;
    const unsigned gmask = T::gbits << (LPR * rs), below = (1u << lane) - 1u;

    // Every moving atom stays at its distance from xb, so the subtree's circles
    // lie in the ball of radius max |x_i - xb| about xb: when that ball is in
    // the grid box for all restarts of the warp, no lookup of this decision
    // needs clamping.  The same loop bounds the subtree in cylindrical
    // coordinates about the axis: axial t = (x - xb).u in [tlo, thi], squared
    // radius in [q2lo, q2hi].
    float rho2 = 0.0f, tlo = INFINITY, thi = -INFINITY, q2lo = INFINITY, q2hi = 0.0f;
    for (int i = b + 1 + g; i < e; i += LPR) {
        const float dx = v.Xx[i * ST + rs] - xbx, dy = v.Xy[i * ST + rs] - xby, dz = v.Xz[i * ST + rs] - xbz;
        const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz)), t = fmaf(u.x, dx, fmaf(u.y, dy, u.z * dz));
        const float q2 = fmaf(-t, t, d2);
        rho2 = fmaxf(rho2, d2);
        tlo = fminf(tlo, t);
        thi = fmaxf(thi, t);
        q2lo = fminf(q2lo, q2);
        q2hi = fmaxf(q2hi, q2);
    }
#pragma unroll
    for (int o = 1; o < LPR; o <<= 1) {
        rho2 = fmaxf(rho2, __shfl_xor_sync(LG_FULL, rho2, o));
        tlo = fminf(tlo, __shfl_xor_sync(LG_FULL, tlo, o));
        thi = fmaxf(thi, __shfl_xor_sync(LG_FULL, thi, o));
        q2lo = fminf(q2lo, __shfl_xor_sync(LG_FULL, q2lo, o));
        q2hi = fmaxf(q2hi, __shfl_xor_sync(LG_FULL, q2hi, o));
    }
    const float rho = sqrtf(rho2) + 1e-2f, lo = 1e-2f, hi = G.gmax - 1e-2f;
    const bool ball_in = xbx + c0 - rho >= lo && xbx + c0 + rho <= hi && xby + c0 - rho >= lo &&
                         xby + c0 + rho <= hi && xbz + c0 - rho >= lo && xbz + c0 + rho <= hi;
#ifndef LG_RT_INSIDE_PATH
#define LG_RT_INSIDE_PATH 1
#endif
    const bool all_in = LG_RT_INSIDE_PATH && __all_sync(LG_FULL, ball_in || !valid);

    // Fixed atoms farther than rho + d_clash from xb can never come within
    // d_clash of a moving atom, and neither can those whose cylindrical
    // coordinates lie outside the subtree's range widened by d_clash: a
    // fixed point's distance to a coaxial circle is at least the distance
    // between the two in the (t, radius) plane.  Each restart keeps a list of
    // the others (the 0.05 A margin covers rounding; dropped atoms have no
    // step within d_clash).
    const float dm = sqrtf(dc2) + 0.05f, rlim = sqrtf(rho2) + dm, rlim2 = rlim * rlim;
    tlo -= dm;
    thi += dm;
    const float rlo = fmaxf(sqrtf(fmaxf(q2lo, 0.0f)) - dm, 0.0f), rhi = sqrtf(q2hi) + dm;
    q2lo = rlo > 0.0f ? rlo * rlo : -INFINITY;  // atoms on the axis (rounding may make q2 < 0) stay in
    q2hi = rhi * rhi;
    int ncnt = 0;  // near fixed atoms of this restart (same in all its lanes)
    for (int jb = 0; jb < nF; jb += LPR) {
        const int jj = jb + g;
        bool nr = false;
        int j = 0;
        if (valid && jj < nF) {
            j = jj < b ? jj : jj + (e - b);
            const float dx = v.Xx[j * ST + rs] - xbx, dy = v.Xy[j * ST + rs] - xby, dz = v.Xz[j * ST + rs] - xbz;
            const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz)), t = fmaf(u.x, dx, fmaf(u.y, dy, u.z * dz));
            const float q2 = fmaf(-t, t, d2);
            nr = d2 < rlim2 && t > tlo && t < thi && q2 > q2lo && q2 < q2hi;
        }
        const unsigned bal = __ballot_sync(LG_FULL, nr);
        if (nr) v.near[rs * v.nstride + LG_IDX(ncnt + __popc(bal & gmask & below), v.nstride, kChkNear)] = (uint8_t)j;
        ncnt += __popc(bal & gmask);
    }
    v.mask[lane] = 0u;
    __syncwarp();
    const int nnear = (int)__reduce_max_sync(LG_FULL, (unsigned)ncnt);

    // Clash pairs of moving atom i (circle C): pairs that can come within
    // d_clash somewhere on the circle are pooled over the warp's restarts and
    // evaluated step by step.
    int pc = 0;  // pooled pairs (warp-uniform)
    auto pool_pairs = [&](int i, const Circle &C) {
        const int excl = (cv.par[i] == b) ? a : -1;  // two bonds apart through the bond itself
        for (int jb = 0; jb < nnear; jb += LPR) {
            if (pc > kPoolCap - 32) flush_pool<LPR>(v, rs, g, pc, cs, sn, dc2);
            const int jj = jb + g;
            PairC q;
            q.near = false;
            if (jj < ncnt) {
                const int j = v.near[rs * v.nstride + jj];
                if (j != excl)
                    q = pair_coeffs(C.px, C.py, C.pz, C.e1x, C.e1y, C.e1z, C.e2x, C.e2y, C.e2z, C.r2, v.Xx[j * ST + rs],
                                    v.Xy[j * ST + rs], v.Xz[j * ST + rs], dc2);
            }
            const unsigned bal = __ballot_sync(LG_FULL, q.near);
            if (q.near) v.pool[LG_IDX(pc + __popc(bal & below), kPoolCap, kChkPool)] = make_float4(q.C, q.A2, q.B2, __int_as_float(rs));
            pc += __popc(bal);
        }
    };

    // Overlap scores of the lane's steps over the moving atoms (in order),
    // and each atom's clash pairs while its cell loads are in flight.  Lanes
    // of an idle slot issue no loads.
    float acc[T::steps];
#pragma unroll
    for (int j = 0; j < T::steps; ++j) acc[j] = 0.0f;
    for (int i = b + 1; i < e; ++i) {
        const Circle C = make_circle(v.Xx[i * ST + rs], v.Xy[i * ST + rs], v.Xz[i * ST + rs], xbx, xby, xbz, u, c0,
                                     G.gmax);
        if (!valid) {
        } else if (all_in) {
#pragma unroll
            for (int j = 0; j < T::steps; ++j) {
                const float3 q = circle_index(C.Px, C.Py, C.Pz, C.e1x, C.e1y, C.e1z, C.e2x, C.e2y, C.e2z, cs[j], sn[j]);
                acc[j] += lookup_in(G, q.x, q.y, q.z);
            }
        } else {
#pragma unroll
            for (int j = 0; j < T::steps; ++j) {
                const float3 q = circle_index(C.Px, C.Py, C.Pz, C.e1x, C.e1y, C.e1z, C.e2x, C.e2y, C.e2z, cs[j], sn[j]);
                acc[j] += lookup_clamped(G, q.x, q.y, q.z);
            }
        }
        if (nnear > 0) pool_pairs(i, C);
    }
    flush_pool<LPR>(v, rs, g, pc, cs, sn, dc2);
    unsigned clash = v.mask[lane];  // bit j: step LPR*j + g clashes
    if (g == 0) clash &= ~1u;        // step 0 (the current pose) is always admissible
    const bool short_lane = T::ragged && g >= T::first_missing;  // no last step
    if (short_lane) clash |= 1u << (T::steps - 1);

    // highest-scoring admissible step of the restart, lowest step on ties
    float bs = -INFINITY;
    int bt = 1024;
#pragma unroll
    for (int j = 0; j < T::steps; ++j)
        if (!((clash >> j) & 1u) && acc[j] > bs) {
            bs = acc[j];
            bt = LPR * j + g;
        }
#pragma unroll
    for (int o = 1; o < LPR; o <<= 1) {
        const float os = __shfl_xor_sync(LG_FULL, bs, o);
        const int ot = __shfl_xor_sync(LG_FULL, bt, o);
        if (better(os, ot, bs, bt)) {
            bs = os;
            bt = ot;
        }
    }
    const int t = (bt > 0 && bt < LG_ANGLE_STEPS) ? bt : 0;
    if (want_rank) {  // steps ranked before the chosen one, admissible or not
        int cnt = 0;
#pragma unroll
        for (int j = 0; j < T::steps; ++j)
            if (!(short_lane && j == T::steps - 1))
                cnt += (acc[j] > bs || (acc[j] == bs && LPR * j + g < t)) ? 1 : 0;
#pragma unroll
        for (int o = 1; o < LPR; o <<= 1) cnt += __shfl_xor_sync(LG_FULL, cnt, o);
        jr = 1 + cnt;
    }
    if (t != 0) {
        const float c = c_cos[t], s = c_sin[t];
        for (int i = b + 1 + g; i < e; i += LPR) {
            const float3 x = rotate_point(v.Xx[i * ST + rs], v.Xy[i * ST + rs], v.Xz[i * ST + rs], xbx, xby, xbz, u,
                                          c, s);
            v.Xx[i * ST + rs] = x.x;
            v.Xy[i * ST + rs] = x.y;
            v.Xz[i * ST + rs] = x.z;
        }
        for (int kk = k + 1 + g; kk < R; kk += LPR)
            if (cv.rch[kk] < e) v.axis[kk * ST + rs] = rotate_vec(v.axis[kk * ST + rs], u, c, s);
    }
    __syncwarp();
    return t;
}

// Rigid greedy moves of the warp's restart slots after torsion pass ps: the
// 13 candidates are scored by sums over atoms in the tile-independent order
// (FP32 overlap lookups of the atoms at their moved positions); the best
// (highest score, lowest candidate) moves the atoms and turns the bond axes.
template <int LPR>
__device__ __forceinline__ bool rigid_moves_rt(const DockArgs &A, float rigid_shift_g, const GridK &Go, const OutDev &O,
                                               const RtView &v, int l, int r, int ps, int N, int R, int rs, int g,
                                               bool valid) {
    constexpr int ST = Rt<LPR>::slots;
    const float c0 = 0.5f * Go.gmax, dg = rigid_shift_g, ca = c_cos[1], sa = c_sin[1];
    bool moved = false;
    for (int j = 0; j < A.rigid_steps; ++j) {
        float cen[3];
        sum4<LPR>(g, N, true, cen, [&](int i, float(&s)[3]) {
            s[0] += v.Xx[i * ST + rs];
            s[1] += v.Xy[i * ST + rs];
            s[2] += v.Xz[i * ST + rs];
        });
        const float cx = cen[0] / (float)N, cy = cen[1] / (float)N, cz = cen[2] / (float)N;
        float Gc[kRigidCandidates];
        sum4<LPR>(g, N, valid, Gc, [&](int i, float(&s)[kRigidCandidates]) {  // idle slots issue no loads
            const float x = v.Xx[i * ST + rs], y = v.Xy[i * ST + rs], z = v.Xz[i * ST + rs];
#pragma unroll
            for (int c = 0; c < kRigidCandidates; ++c) {
                const float3 q = rigid_candidate(c, x, y, z, cx, cy, cz, dg, ca, sa);
                s[c] += lookup_clamped(Go, q.x + c0, q.y + c0, q.z + c0);
            }
        });
        float bG = -INFINITY;
        int bC = kRigidCandidates;
#pragma unroll
        for (int c = 0; c < kRigidCandidates; ++c)
            if (Gc[c] > bG) {  // ascending candidates: ties keep the lower one
                bG = Gc[c];
                bC = c;
            }
        if (valid && g == 0 && O.restart_rigid)
            O.restart_rigid[(((size_t)l * A.S + r) * A.P + ps) * A.rigid_steps + j] = (uint8_t)bC;
        __syncwarp();
        moved = moved || bC != 0;
        if (bC != 0) {
            for (int i = g; i < N; i += LPR) {
                const float3 y = rigid_candidate(bC, v.Xx[i * ST + rs], v.Xy[i * ST + rs], v.Xz[i * ST + rs], cx, cy,
                                                 cz, dg, ca, sa);
                v.Xx[i * ST + rs] = y.x;
                v.Xy[i * ST + rs] = y.y;
                v.Xz[i * ST + rs] = y.z;
            }
            for (int k = g; k < R; k += LPR) v.axis[k * ST + rs] = rigid_candidate_vec(bC, v.axis[k * ST + rs], ca, sa);
        }
        __syncwarp();
    }
    return moved;
}

// kRank: pose ranking on; kRigid: rigid refinement on; kTrace: decision
// ranks recorded (separate instantiations, so the plain best-restart form
// carries none of their code); LPR: lanes per restart of the warp's tile
template <bool kRank, bool kRigid, bool kTrace, int LPR>
__device__ __forceinline__ void dock_ligand_rt(const DockArgs &A, const PocketDev &Pk, const OutDev &O, const LigSrc &Q, int l,
                                               char *sm) {
    using T = Rt<LPR>;
    constexpr int ST = T::slots;
    if (O.status[l] != LG_OK) return;  // rejected by the preparation kernel (uniform)
    const Layout &Ly = A.ly;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
    const int rs = lane / LPR, g = lane % LPR;
    const CtaView cv = cta_view(sm, Ly);
    const RtView v = rt_view<LPR>(sm, Ly, A.lrt, warp);
    const BatchDev &B = Q.batch;
    const int a0 = B.atom_off[l], N = B.atom_off[l + 1] - a0;
    const int r0 = B.rot_off[l], R = B.rot_off[l + 1] - r0;
    const int S = A.S, P = A.P, PR = P * R;
    stage_ligand(A, B, Pk, cv, l, a0, N, r0, R);
    __syncthreads();

    float cs[T::steps], sn[T::steps];
#pragma unroll
    for (int j = 0; j < T::steps; ++j) {
        const int t = LPR * j + g < LG_ANGLE_STEPS ? LPR * j + g : 0;  // a ragged round's missing step: step 0's angle
        cs[j] = c_cos[t];
        sn[j] = c_sin[t];
    }
    const uint64_t uid = B.uid[l];
    const uint2 key = make_uint2(A.seed_lo, A.seed_hi);
    const GridK Go = grid_k(Pk, Pk.cell_o), Gve = grid_k(Pk, Pk.cell_ve);
    // Restart streaming: warp w owns restarts w, w + W, w + 2W, ... and runs
    // them through its restart slots.  All slots take the same bond at the
    // same time, pass after pass; a slot whose restart has finished (P passes,
    // or converged: R decisions in a row without a move, or with rigid moves a
    // pass without one -- every later decision would repeat step 0) is emptied
    // at the end of the pass and refilled with the warp's next restart, which
    // starts its first pass with the others' next one.  A restart's arithmetic
    // does not depend on its slot, so results are those of restarts run alone.
    int r = warp + W * rs;  // this slot's restart (-1: idle)
    if (r >= S) r = -1;
    int qnext = ST;         // next index into the warp's restart list (uniform)
    int pc = 0;             // passes this slot's restart has completed
    int zrun = 0;           // its decisions in a row without a move
    bool movedp = true;     // whether it moved in its last pass
    bool fresh = true;      // slot needs its restart's initial pose (an idle slot takes restart 0's, never used)
    double bestE = INFINITY;
    int bestR = -1;
    for (;;) {
        // 1. initial pose of newly filled slots (the lanes of a slot split atoms and bonds)
        if (fresh) {
            const Pose pose = restart_pose(uid, (uint32_t)(r >= 0 ? r : 0), key, Pk.n_pp);
            const float4 pp = __ldg(Pk.pp + pose.pp);
            for (int i = g; i < N; i += LPR) {
                const float3 x = rot_add(pose.R, cv.d0x[i], cv.d0y[i], cv.d0z[i], pp.x, pp.y, pp.z);
                v.Xx[i * ST + rs] = x.x;
                v.Xy[i * ST + rs] = x.y;
                v.Xz[i * ST + rs] = x.z;
            }
            for (int k = g; k < R; k += LPR) {
                const float4 d = cv.dv[k];
                const float3 w = rot_vec(pose.R, d.x, d.y, d.z);
                v.axis[k * ST + rs] = make_float4(w.x, w.y, w.z, 0.0f);
            }
            fresh = false;
        }
        __syncwarp();
        // 2. finished restarts: remaining decisions are step 0; score, outputs, best
        const bool active = r >= 0;
        const bool conv = kRigid ? (pc > 0 && !movedp) : (zrun >= R);
        const bool done = active && (pc >= P || conv);
        if (__any_sync(LG_FULL, done)) {
            if (done) {
                for (int q = pc * R + g; q < PR; q += LPR) v.tcur[q * ST + rs] = 0;
                if (kTrace && g == 0) {  // skipped passes repeat the last one, marked skipped
                    uint8_t *dr = O.decision_rank + (size_t)S * P * r0 + (size_t)r * PR;
                    for (int q = pc * R; q < PR; ++q) dr[q] = dr[q - R] | kRankSkipped;
                }
                if (kRigid && g == 0 && O.restart_rigid)
                    for (int q = pc * A.rigid_steps; q < P * A.rigid_steps; ++q)
                        O.restart_rigid[((size_t)l * S + r) * P * A.rigid_steps + q] = 0;
            }
            __syncwarp();
            // pose score: FP32 per-atom terms, FP64 sums in the tile-independent order
            double Es[1];
            sum4<LPR>(g, N, done, Es, [&](int i, double(&s)[1]) {
                const float2 wq = cv.wq[i];
                s[0] += (double)atom_energy(Pk, Gve, v.Xx[i * ST + rs], v.Xy[i * ST + rs], v.Xz[i * ST + rs], wq.x,
                                            wq.y);
            });
            const double E = Es[0];
            if (done) {
                if (O.restart_score && g == 0) O.restart_score[(size_t)l * S + r] = E;
                if (O.restart_tors)
                    for (int t = g; t < PR; t += LPR)
                        O.restart_tors[(size_t)S * P * r0 + (size_t)r * PR + t] = v.tcur[t * ST + rs];
                if (kRank) {  // keep the restart for the ranking step
                    const int slot = rank_slot(A, blockIdx.x);
                    float *x = A.scr.rk_pose + rk_pose_off(A, slot, r);
                    for (int i = g; i < N; i += LPR) {
                        x[3 * i] = v.Xx[i * ST + rs];
                        x[3 * i + 1] = v.Xy[i * ST + rs];
                        x[3 * i + 2] = v.Xz[i * ST + rs];
                    }
                    for (int t = g; t < PR; t += LPR)
                        A.scr.rk_tors[((size_t)slot * S + r) * P * Ly.rmax + t] = v.tcur[t * ST + rs];
                    if (g == 0) A.scr.rk_E[(size_t)slot * S + r] = E;
                }
            }
            if (kRank) {  // the restart's geometric score and centroid for the ranking step
                float gq[4];
                sum4<LPR>(g, N, done, gq, [&](int i, float(&s)[4]) {
                    const float x = v.Xx[i * ST + rs], y = v.Xy[i * ST + rs], z = v.Xz[i * ST + rs];
                    s[0] += lookup_clamped(Go, x + Pk.c0, y + Pk.c0, z + Pk.c0);
                    s[1] += x;
                    s[2] += y;
                    s[3] += z;
                });
                if (done && g == 0) {
                    const size_t q = (size_t)rank_slot(A, blockIdx.x) * S + r;
                    A.scr.rk_G[q] = gq[0];
                    A.scr.rk_cen[3 * q] = gq[1];
                    A.scr.rk_cen[3 * q + 1] = gq[2];
                    A.scr.rk_cen[3 * q + 2] = gq[3];
                }
            }
            // best of the finished restarts (lowest E, then lowest restart), then of the warp
            double te = done ? E : INFINITY;
            int tr = done ? r : 0x7fffffff, ts = rs;
#pragma unroll
            for (int o = LPR; o < 32; o <<= 1) {
                const double oe = __shfl_xor_sync(LG_FULL, te, o);
                const int orr = __shfl_xor_sync(LG_FULL, tr, o), os = __shfl_xor_sync(LG_FULL, ts, o);
                if (oe < te || (oe == te && orr < tr)) {
                    te = oe;
                    tr = orr;
                    ts = os;
                }
            }
            if (tr != 0x7fffffff && (bestR < 0 || te < bestE || (te == bestE && tr < bestR))) {
                bestE = te;
                bestR = tr;
                for (int t = lane; t < PR; t += 32) v.tbest[t] = v.tcur[t * ST + ts];
                if (Ly.want_pose)
                    for (int i = lane; i < N; i += 32) {
                        v.Bx[i] = v.Xx[i * ST + ts];
                        v.By[i] = v.Xy[i * ST + ts];
                        v.Bz[i] = v.Xz[i * ST + ts];
                    }
            }
            __syncwarp();
            // refill the finished slots, in slot order, from the warp's restart list
            const unsigned dm = __ballot_sync(LG_FULL, done && g == 0);
            if (done) {
                const int j = qnext + __popc(dm & ((1u << (LPR * rs)) - 1u));
                const int rn = warp + W * j;
                r = rn < S ? rn : -1;
                pc = 0;
                zrun = 0;
                movedp = true;
                fresh = r >= 0;
            }
            qnext += __popc(dm);
            continue;  // initial poses first
        }
        if (!__any_sync(LG_FULL, active)) break;
        // 3. one greedy pass over the torsional bonds for every active slot
        movedp = false;
        for (int k = 0; k < R; ++k) {
            // a restart R zero decisions in a row into the pass sequence repeats
            // them from here on (step 0, no move): its lanes skip the work
            const bool sv = kRigid || zrun < R;
            int jr;
            const int t = sweep_bond_rt<LPR>(Q.dc2g, Go, cv, v, N, R, k, rs, g, active && sv, cs, sn, kTrace, jr);
            if (active && g == 0) {
                v.tcur[LG_IDX(pc * R + k, P * Ly.rmax, kChkDecision) * ST + rs] = (uint8_t)t;
                if (kTrace) {  // a skipped decision repeats the bond's previous one
                    uint8_t *dr = O.decision_rank + (size_t)S * P * r0 + (size_t)r * PR + pc * R + k;
                    *dr = sv ? (uint8_t)jr : (uint8_t)(dr[-R] | kRankSkipped);
                }
            }
            movedp = movedp || t != 0;
            zrun = t != 0 ? 0 : zrun + 1;
            if (!kRigid && !__any_sync(LG_FULL, active && zrun < R)) {  // every active restart converged
                if (active)
                    for (int q = pc * R + k + 1 + g; q < (pc + 1) * R; q += LPR) v.tcur[q * ST + rs] = 0;
                if (kTrace && active && g == 0) {
                    uint8_t *dr = O.decision_rank + (size_t)S * P * r0 + (size_t)r * PR;
                    for (int q = pc * R + k + 1; q < (pc + 1) * R; ++q) dr[q] = dr[q - R] | kRankSkipped;
                }
                break;
            }
        }
        if (kRigid) movedp = rigid_moves_rt<LPR>(A, Q.rigid_shift_g, Go, O, v, l, r, pc, N, R, rs, g, active) || movedp;
        if (active) pc++;
        __syncwarp();
    }
    if (kRank) {
        __syncthreads();
        rank_finish(A, Pk, O, Q.thr2g, l, rank_slot(A, blockIdx.x), a0, N, r0, PR, sm + Ly.cta_bytes);
        return;
    }
    if (lane == 0) {
        cv.wE[warp] = bestE;
        cv.wR[warp] = bestR;
    }
    finish_ligand(A, Pk, O, cv, l, a0, N, r0, PR, [&](int w, const float *&Bx, const float *&By, const float *&Bz,
                                                     const uint8_t *&tb) {
        const RtView bv = rt_view<LPR>(sm, Ly, A.lrt, w);
        Bx = bv.Bx;
        By = bv.By;
        Bz = bv.Bz;
        tb = bv.tbest;
    });
}

// Persistent: CTAs pull ligands from a device counter in cost order.  The
// launch bounds keep 128 registers per thread for every tile (warps per CTA
// up to Rt<LPR>::max_warps).
#ifndef LG_RT_MIN_BLOCKS
#define LG_RT_MIN_BLOCKS 4
#endif
template <bool kRank, bool kRigid, bool kTrace, int LPR>
__global__ void __launch_bounds__(32 * Rt<LPR>::max_warps, 4 * LG_RT_MIN_BLOCKS / Rt<LPR>::max_warps)
    k_dock_batched(const __grid_constant__ DockArgs A) {
    extern __shared__ __align__(16) char sm[];
    __shared__ int s_lig;
    for (;;) {
        if (threadIdx.x == 0) {  // next ligand of the launch's range of the cost order, or -1
            int first = 0, count = A.batch.L;
            if (A.cls_off) {  // one size class
                first = A.cls_off[2 - A.cls];
                count = A.cls_off[3 - A.cls] - first;
            }
            int stride = 1;
            if (A.item_cap > 0 && count > A.item_cap) {  // autotuning trial: an even sample of the range
                stride = count / A.item_cap;
                count = A.item_cap;
            }
            const int item = atomicAdd(A.work_counter, 1);
            const int at = first + item * stride;
            s_lig = item < count ? (A.order ? A.order[at] : at) : -1;
        }
        __syncthreads();
        const int l = s_lig;
        __syncthreads();
        if (l < 0) break;
        dock_ligand_rt<kRank, kRigid, kTrace, LPR>(A, A.pocket, A.out, launch_src(A), l, sm);
    }
}

// Several pockets (MultiDev): work items are (pocket, ligand) pairs; the
// docking code is the single-pocket code with the item's pocket and outputs.
// The preparation kernel validated every ligand once and wrote its status to
// the first pocket's outputs; the other pockets' outputs get the same status
// here.
template <bool kRank, bool kRigid>
__global__ void __launch_bounds__(128, LG_RT_MIN_BLOCKS) k_dock_multi(const __grid_constant__ DockArgs A,
                                                                       const __grid_constant__ MultiDev M) {
    extern __shared__ __align__(16) char sm[];
    __shared__ int s_item;
    const int L = A.batch.L;
    int items = (M.pocket_major && !M.lig_pocket) ? M.np * L : L;
    int stride = 1;
    if (A.item_cap > 0) {  // autotuning trial: an even sample of the ligands (of the first pocket when
                           // pocket-major, as the full launch keeps one pocket's grids in L2 at a time)
        const int span = min(items, L);
        stride = max(1, span / A.item_cap);
        items = min(A.item_cap, span);
    }
    auto dock_one = [&](int p, int l) {
        const OutDev &O = M.out[p];
        if (p > 0) {
            if (threadIdx.x == 0) {
                const int st = M.out[0].status[l];
                O.status[l] = st;
                if (st != LG_OK) {
                    O.score[l] = __longlong_as_double(0x7ff8000000000000ll);
                    O.best_restart[l] = -1;
                }
            }
            __syncthreads();
        }
        dock_ligand_rt<kRank, kRigid, false, 4>(A, M.pk[p], O, launch_src(A), l, sm);
        __syncthreads();
    };
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(A.work_counter, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= items) break;
        const int at = item * stride;
        if (M.lig_pocket) {  // one pocket per ligand
            const int l = A.order ? A.order[at] : at;
            dock_ligand_rt<kRank, kRigid, false, 4>(A, M.pk[M.lig_pocket[l]], A.out, launch_src(A), l, sm);
            __syncthreads();
        } else if (M.pocket_major) {
            const int p = at / L, i = at - p * L;
            dock_one(p, A.order ? A.order[i] : i);
        } else {
            const int l = A.order ? A.order[at] : at;
            for (int p = 0; p < M.np; ++p) dock_one(p, l);
        }
    }
}

// ================================================================== flattening
// Ligand pre-processing (paper Sec. 3.1, step 1; no pocket): the greedy sweep
// with the sum of all pairwise atom distances as its objective.  One warp per
// ligand, positions centroid-relative in A (FP32).  Lanes own torsion steps
// (lane t: step t, lanes 0..3 also steps 32..35).  Only the (moving, fixed)
// pairs change with the step: their distance on the step's circle point is
//     |x_i(theta) - x_j| = sqrt(C + A2 cos(theta) + B2 sin(theta)),
// with the pair coefficients built once per decision, 128 pairs at a time by
// the lanes and read back by broadcast.  Per step, distances are summed in FP32
// within a 128-pair chunk, the chunks in FP64 and the lanes' totals in FP32;
// the clash rule of the sweep (pairs at least three bonds apart, at least
// d_clash) decides admissibility;
// the admissible step with the largest sum wins, the lowest step on ties.
__global__ void __launch_bounds__(32 * kFlatWarps) k_flatten(const __grid_constant__ FlatArgs F) {
    extern __shared__ __align__(16) char sm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int l = blockIdx.x * kFlatWarps + warp;
    if (l >= F.batch.L) return;  // warp-uniform; no CTA barriers below
    const BatchDev &B = F.batch;
    const int a0 = B.atom_off[l], N = B.atom_off[l + 1] - a0;
    if (F.status[l] != LG_OK) {  // rejected by the preparation kernel: coordinates pass through
        for (int i = lane; i < N && i < LG_MAX_ATOMS; i += 32) {
            F.xyz[3 * (size_t)(a0 + i)] = B.x[a0 + i];
            F.xyz[3 * (size_t)(a0 + i) + 1] = B.y[a0 + i];
            F.xyz[3 * (size_t)(a0 + i) + 2] = B.z[a0 + i];
        }
        if (F.dsum && lane == 0) F.dsum[l] = __longlong_as_double(0x7ff8000000000000ll);
        return;
    }
    const int nm = F.nmax;
    char *wb = sm + (size_t)warp * flat_warp_bytes(nm);
    float *Xx = (float *)wb, *Xy = Xx + nm, *Xz = Xy + nm;
    int *par = (int *)(wb + lg_align16(12 * nm));
    float4 *circ = (float4 *)(wb + lg_align16(12 * nm) + lg_align16(4 * nm));  // [nm][3]: (p, r2), e1, e2
    float4 *chunk = circ + 3 * nm;                                              // [kFlatChunk] (C, A2, B2, checked)
    const int r0 = B.rot_off[l], R = B.rot_off[l + 1] - r0;
    const double cx = F.centroid[3 * l], cy = F.centroid[3 * l + 1], cz = F.centroid[3 * l + 2];
    for (int i = lane; i < N; i += 32) {
        Xx[i] = (float)((double)B.x[a0 + i] - cx);
        Xy[i] = (float)((double)B.y[a0 + i] - cy);
        Xz[i] = (float)((double)B.z[a0 + i] - cz);
        par[i] = B.parent[a0 + i];
    }
    __syncwarp();
    // lanes: 4 step groups (g: steps g, g+4, ..., g+32) x 8 pair groups (pg)
    const int g = lane & 3, pg = lane >> 2;
    float cs[kStepsPerLane], sn[kStepsPerLane];
#pragma unroll
    for (int j = 0; j < kStepsPerLane; ++j) {
        cs[j] = c_cos[4 * j + g];
        sn[j] = c_sin[4 * j + g];
    }
    // R decisions in a row without a move (one round over every bond) leave
    // the state as they saw it: every later decision repeats one of them, so
    // the sweep stops and records step 0 for the rest (exact)
    int zrun = 0;
    bool converged = false;
    for (int ps = 0; ps < F.P && !converged; ++ps)
        for (int k = 0; k < R; ++k) {
            const int b = B.rot_child[r0 + k], a = par[b], e = F.rot_end[(size_t)l * F.rmax_lim + k];
            const float xbx = Xx[b], xby = Xy[b], xbz = Xz[b];
            const float3 u = unit_axis(make_float4(xbx - Xx[a], xby - Xy[a], xbz - Xz[a], 0.0f));
            for (int i = b + 1 + lane; i < e; i += 32) {
                const Circle C = make_circle(Xx[i], Xy[i], Xz[i], xbx, xby, xbz, u, 0.0f, 0.0f);
                circ[3 * i] = make_float4(C.px, C.py, C.pz, C.r2);
                circ[3 * i + 1] = make_float4(C.e1x, C.e1y, C.e1z, 0.0f);
                circ[3 * i + 2] = make_float4(C.e2x, C.e2y, C.e2z, 0.0f);
            }
            __syncwarp();
            const int m = e - b - 1, nf = N - (e - b);
            const int total = m * nf;
            double D[kStepsPerLane];
            float mn[kStepsPerLane];
#pragma unroll
            for (int j = 0; j < kStepsPerLane; ++j) {
                D[j] = 0.0;
                mn[j] = INFINITY;
            }
            for (int q0 = 0; q0 < total; q0 += kFlatChunk) {
#pragma unroll
                for (int u = 0; u < kFlatChunk / 32; ++u) {
                    const int q = q0 + 32 * u + lane;
                    if (q < total) {
                        const int i = b + 1 + q / nf, jj = q - (q / nf) * nf;
                        const int j = jj < b ? jj : jj + (e - b);
                        const float4 pc = circ[3 * i], e1 = circ[3 * i + 1], e2 = circ[3 * i + 2];
                        const PairC pq = pair_coeffs(pc.x, pc.y, pc.z, e1.x, e1.y, e1.z, e2.x, e2.y, e2.z, pc.w, Xx[j],
                                                     Xy[j], Xz[j], F.dc2);
                        const bool checked = !(j == a && par[i] == b);  // the one pair closer than 3 bonds
                        chunk[32 * u + lane] = make_float4(pq.C, pq.A2, pq.B2, checked ? 1.0f : 0.0f);
                    }
                }
                __syncwarp();
                const int n = min(kFlatChunk, total - q0);
                float acc[kStepsPerLane];
#pragma unroll
                for (int j = 0; j < kStepsPerLane; ++j) acc[j] = 0.0f;
                for (int t = pg; t < n; t += 8) {  // the lane's pairs of the chunk, its 9 steps each
                    const float4 cf = chunk[t];
#pragma unroll
                    for (int j = 0; j < kStepsPerLane; ++j) {
                        const float d = fmaf(cf.z, sn[j], fmaf(cf.y, cs[j], cf.x));
                        // d * rsqrt(d): the hardware reciprocal square root
                        // (about 2 ulp) instead of a correctly rounded sqrt;
                        // sums of positive terms keep that relative error
                        acc[j] += d > 0.0f ? d * rsqrtf(d) : 0.0f;
                        if (cf.w != 0.0f) mn[j] = fminf(mn[j], d);
                    }
                }
#pragma unroll
                for (int j = 0; j < kStepsPerLane; ++j) D[j] += (double)acc[j];
                __syncwarp();
            }
            // totals over the 8 pair groups (FP32: eight terms, ~1e-7
            // relative), then the best admissible step of the lane and of the
            // warp (larger sum, then lower step)
            float bd = -INFINITY;
            int bt = 1024;
#pragma unroll
            for (int j = 0; j < kStepsPerLane; ++j) {
                float dj = (float)D[j];
#pragma unroll
                for (int o = 4; o < 32; o <<= 1) {
                    dj += __shfl_xor_sync(LG_FULL, dj, o);
                    mn[j] = fminf(mn[j], __shfl_xor_sync(LG_FULL, mn[j], o));
                }
                const int t = 4 * j + g;
                if ((t == 0 || mn[j] >= F.dc2) && dj > bd) {
                    bd = dj;
                    bt = t;
                }
            }
#pragma unroll
            for (int o = 1; o < 4; o <<= 1) {
                const float od = __shfl_xor_sync(LG_FULL, bd, o);
                const int ot = __shfl_xor_sync(LG_FULL, bt, o);
                if (od > bd || (od == bd && ot < bt)) {
                    bd = od;
                    bt = ot;
                }
            }
            if (F.tors && lane == 0) F.tors[(size_t)F.P * r0 + ps * R + k] = (uint8_t)bt;
            if (bt != 0) {
                const float c = c_cos[bt], sn = c_sin[bt];
                for (int i = b + 1 + lane; i < e; i += 32) {
                    const float4 pc = circ[3 * i], e1 = circ[3 * i + 1], e2 = circ[3 * i + 2];
                    Xx[i] = fmaf(e2.x, sn, fmaf(e1.x, c, pc.x));
                    Xy[i] = fmaf(e2.y, sn, fmaf(e1.y, c, pc.y));
                    Xz[i] = fmaf(e2.z, sn, fmaf(e1.z, c, pc.z));
                }
            }
            __syncwarp();
            zrun = bt != 0 ? 0 : zrun + 1;
            if (zrun >= R) {
                if (F.tors)
                    for (int q = ps * R + k + 1 + lane; q < F.P * R; q += 32) F.tors[(size_t)F.P * r0 + q] = 0;
                converged = true;
                break;
            }
        }
    // outputs: coordinates in the input frame and the final sum of distances
    for (int i = lane; i < N; i += 32) {
        F.xyz[3 * (size_t)(a0 + i)] = (float)((double)Xx[i] + cx);
        F.xyz[3 * (size_t)(a0 + i) + 1] = (float)((double)Xy[i] + cy);
        F.xyz[3 * (size_t)(a0 + i) + 2] = (float)((double)Xz[i] + cz);
    }
    if (F.dsum) {
        double D = 0.0;
        for (int i = lane; i < N; i += 32)
            for (int j = i + 1; j < N; ++j) {
                const float dx = Xx[i] - Xx[j], dy = Xy[i] - Xy[j], dz = Xz[i] - Xz[j];
                D += (double)sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
            }
        D = warp_sum_d(D);
        if (lane == 0) F.dsum[l] = D;
    }
}

// ================================================================== preparation and sorting
// One thread per ligand: validates the ligand (sizes within the limits,
// parent[0] = -1, parent[i] < i, contiguous subtrees -- subtree size equals
// end - start --, types, finite coordinates, torsional children strictly
// ascending in [1, N-1]), writes the end of every torsional child's subtree,
// the centroid (FP64) and the ligand's status; with `sort` it also files the
// ligand into a log-scale cost bucket (4 per octave) of
//   cost ~ restarts * (passes * 36 * sum of moving atoms + 8 * atoms + 64):
// 4 buckets per octave, or (sort_classes) the size class and 2 buckets per
// octave within it (rejected ligands: class 0).
// Where the preparation reads a ligand's atoms: the batch in global memory,
// or a copy of them in shared memory.
struct AtomsGlobal {
    const BatchDev &B;
    int a0, r0;
    __device__ float x(int i) const { return B.x[a0 + i]; }
    __device__ float y(int i) const { return B.y[a0 + i]; }
    __device__ float z(int i) const { return B.z[a0 + i]; }
    __device__ int parent(int i) const { return B.parent[a0 + i]; }
    __device__ int type(int i) const { return B.type[a0 + i]; }
    __device__ int rot_child(int k) const { return B.rot_child[r0 + k]; }
};

struct AtomsShared {
    const float *xs, *ys, *zs;
    const int16_t *par, *rc;
    const uint8_t *ty;
    __device__ float x(int i) const { return xs[i]; }
    __device__ float y(int i) const { return ys[i]; }
    __device__ float z(int i) const { return zs[i]; }
    __device__ int parent(int i) const { return par[i]; }
    __device__ int type(int i) const { return ty[i]; }
    __device__ int rot_child(int k) const { return rc[k]; }
};

// The preparation of ligand l (one thread): validation, the end of every
// torsional child's subtree and the FP64 centroid (atoms summed in order),
// written at entry li of the scratch; the ligand's status (and, when
// rejected, its score and best restart) in O.  Returns whether the ligand is
// valid and, in msum, the sum of its moving atoms.
template <class Src>
__device__ bool prep_core(const DockArgs &A, const Src &at, int N, int R, const OutDev &O, int l, size_t li, long &msum) {
    bool ok = N >= 1 && N <= A.nmax_lim && R >= 0 && R <= A.rmax_lim;
    msum = 0;
    if (ok) {
        int endv[LG_MAX_ATOMS], size[LG_MAX_ATOMS];
        ok = at.parent(0) == -1;
        double sx = 0.0, sy = 0.0, sz = 0.0;
        for (int i = 0; i < N && ok; i++) {
            endv[i] = i + 1;
            size[i] = 1;
            const float x = at.x(i), y = at.y(i), z = at.z(i);
            if (i > 0) {
                const int p = at.parent(i);
                ok = p >= 0 && p < i;
            }
            ok = ok && at.type(i) < LG_NUM_TYPES && isfinite(x) && isfinite(y) && isfinite(z);
            sx += x;
            sy += y;
            sz += z;
        }
        if (ok) {
            for (int i = N - 1; i >= 1; i--) {
                const int p = at.parent(i);
                endv[p] = max(endv[p], endv[i]);
                size[p] += size[i];
            }
            for (int i = 0; i < N && ok; i++) ok = size[i] == endv[i] - i;
            int prev = 0;
            for (int k = 0; k < R && ok; k++) {
                const int b = at.rot_child(k);
                ok = b >= 1 && b < N && b > prev;
                if (ok) {
                    A.scr.rot_end[li * A.rmax_lim + k] = (int16_t)endv[b];
                    msum += endv[b] - b - 1;
                    prev = b;
                }
            }
        }
        if (ok) {
            A.scr.centroid[3 * li] = sx / N;
            A.scr.centroid[3 * li + 1] = sy / N;
            A.scr.centroid[3 * li + 2] = sz / N;
        }
    }
    O.status[l] = ok ? LG_OK : LG_EINVAL;
    if (!ok) {
        O.score[l] = __longlong_as_double(0x7ff8000000000000ll);
        O.best_restart[l] = -1;
    }
    return ok;
}

__device__ bool prep_one(const DockArgs &A, const BatchDev &B, const OutDev &O, int l, size_t li, long &msum) {
    const int a0 = B.atom_off[l], N = B.atom_off[l + 1] - a0;
    const int r0 = B.rot_off[l], R = B.rot_off[l + 1] - r0;
    return prep_core(A, AtomsGlobal{B, a0, r0}, N, R, O, l, li, msum);
}

// The preparation of ligand l by a CTA: its atoms are copied to shared memory
// (`buf`, room for the atom and torsion maxima) by every thread, then thread
// 0 prepares it from there (the same steps and order as prep_one).  Ends
// after a CTA barrier.
__device__ __noinline__ void prep_cta(const DockArgs &A, const BatchDev &B, const OutDev &O, int l, size_t li, char *buf) {
    const int a0 = B.atom_off[l], N = B.atom_off[l + 1] - a0;
    const int r0 = B.rot_off[l], R = B.rot_off[l + 1] - r0;
    const int nm = (A.nmax_lim + 3) & ~3;
    float *xs = (float *)buf, *ys = xs + nm, *zs = ys + nm;
    int16_t *par = (int16_t *)(zs + nm), *rc = par + nm;
    uint8_t *ty = (uint8_t *)(rc + ((A.rmax_lim + 1) & ~1));
    const bool fits = N >= 1 && N <= A.nmax_lim && R >= 0 && R <= A.rmax_lim;
    if (fits) {
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            xs[i] = B.x[a0 + i];
            ys[i] = B.y[a0 + i];
            zs[i] = B.z[a0 + i];
            par[i] = B.parent[a0 + i];
            ty[i] = B.type[a0 + i];
        }
        for (int k = threadIdx.x; k < R; k += blockDim.x) rc[k] = B.rot_child[r0 + k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long msum;
        prep_core(A, AtomsShared{xs, ys, zs, par, rc, ty}, N, R, O, l, li, msum);
    }
    __syncthreads();
}

__global__ void k_prep(const __grid_constant__ DockArgs A, int sort) {
    __shared__ int sh[kSortBuckets];
    if (sort)
        for (int t = threadIdx.x; t < kSortBuckets; t += blockDim.x) sh[t] = 0;
    __syncthreads();
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l < A.batch.L) {
        const int N = A.batch.atom_off[l + 1] - A.batch.atom_off[l];
        long msum = 0;
        const bool ok = prep_one(A, A.batch, A.out, l, (size_t)l, msum);
        if (sort) {
            const double cost = ok ? (double)A.S * ((double)A.P * 36.0 * (double)msum + 8.0 * N + 64.0) : 1.0;
            int key;
            if (A.sort_classes) {  // size class, then 2 buckets per octave of cost
                const int cb = max(0, min(kCostBuckets - 1, (int)(2.0 * log2(cost)) - 16));
                key = size_class(ok ? N : 1) * kCostBuckets + cb;
            } else {  // 4 buckets per octave of cost
                key = max(0, min(kSortBuckets - 1, (int)(4.0 * log2(cost)) - 32));
            }
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
__global__ void k_sort_scan(int32_t *hist, int L) {
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
    __syncwarp();
    if (lane == 0) {  // class boundaries: a class starts at the offset of its costliest bucket
        int32_t *co = hist + kSortBuckets + kSizeClasses + 1;
        for (int c = kSizeClasses - 1; c >= 0; --c) co[kSizeClasses - 1 - c] = hist[c * kCostBuckets + kCostBuckets - 1];
        co[kSizeClasses] = L;
    }
}

__global__ void k_sort_scatter(int L, const int32_t *keys, int32_t *hist, int32_t *order) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l < L) order[atomicAdd(&hist[keys[l]], 1)] = l;
}

// ================================================================== device-resident serving loop
__device__ __forceinline__ uint64_t ld_acquire_u64(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_sys_u64(uint64_t *p, uint64_t v) {
    asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// The next ligand of the CTA (thread 0): the one it holds, else one that CTAs
// of an earlier launch left claimed but undocked (CTA b takes held[b],
// held[b + grid], ...: the earlier launch may have had more CTAs; hk is the
// next of these slots), else a new one by fetch-and-add on `next`; it is
// docked once published (below `tail`).  Returns its index; or -1 when the
// host asked the loop to stop or another CTA reached the idle limit (the
// launch then ends as a whole, so the host relaunches it at full width and
// nothing waits on CTAs that have left), or -2 when the CTA has waited the
// idle limit itself.  On -1 / -2 `held` keeps an unpublished ligand for the
// next launch.  Every wait here ends.
__device__ __noinline__ long long loop_claim(const LoopArgs &S, long long &held, int &hk, uint64_t &deadline) {
    while (held < 0 && hk < S.held_n) {
        const long long h = S.held[hk];
        S.held[hk] = -1;
        hk += (int)gridDim.x;
        if (h >= 0) {
            held = h;
            deadline = global_ns() + S.idle_ns;
        }
    }
    if (held < 0) {
        // once the launch is stopping or closing no CTA claims a new ligand,
        // so every CTA leaves after the one it holds and the launch ends
        // promptly; the ligands left unclaimed wait for the next launch
        if (ld_acquire_u32(&S.ctl->stop) || ld_acquire_u32(&S.ctl->closing)) return -1;
        held = (long long)atomicAdd((unsigned long long *)&S.ctl->next, 1ull);
        deadline = global_ns() + S.idle_ns;
    }
    unsigned nap = 64;
    for (int poll = 0;; ++poll) {
        if ((uint64_t)held < ld_acquire_u64(&S.ctl->tail)) {
            const long long n = held;
            held = -1;
            return n;
        }
        if ((poll & 7) == 0 && (ld_acquire_u32(&S.ctl->stop) || ld_acquire_u32(&S.ctl->closing))) return -1;
        if (global_ns() > deadline) {
            atomicExch(&S.ctl->closing, 1u);
            return -2;
        }
        __nanosleep(nap);
        nap = nap < 4096 ? 2 * nap : 4096;
    }
}

// The descriptor of ligand `item` (thread 0): scanned forward from `hint`
// (descriptors are published in ligand order).  A slot whose sequence number
// is not the one looked for was recycled, so its request is complete and its
// ligands lie below `item`; a descriptor is read between two reads of its
// sequence number (the host invalidates it before rewriting the body).
// Returns false when no descriptor holds the item within 2 * ring steps.
__device__ __noinline__ bool loop_find(const LoopArgs &S, long long item, uint64_t &hint, uint64_t &seq, uint64_t &first, int &L,
                          int &slot, int &pocket) {
    for (int step = 0; step < 2 * S.ring; ++step) {
        const uint64_t head = ld_acquire_u64(&S.ctl->head_seq);
        if (head > hint) hint = head;
        const LoopDesc *d = S.desc + LG_IDX(hint % (uint64_t)S.ring, S.ring, kChkRing);
        if (ld_acquire_u64(&d->seq) != hint) {
            ++hint;
            continue;
        }
        const uint64_t f = d->first;
        const int n = d->L, sl = d->slot, pk = d->pocket;
        __threadfence();
        if (ld_acquire_u64(&d->seq) != hint) {  // rewritten while read: it was complete
            ++hint;
            continue;
        }
        if ((uint64_t)item >= f + (uint64_t)n) {
            ++hint;
            continue;
        }
        if ((uint64_t)item < f || pk < 0 || pk >= S.np) return false;
        seq = hint;
        first = f;
        L = n;
        slot = sl;
        pocket = pk;
        return true;
    }
    return false;
}

// A ligand of request `seq` (L ligands) is docked: its outputs are made
// visible to the host before it is counted, and the CTA that counts the
// request's last ligand raises the request's completion flag (thread 0).
__device__ __noinline__ void loop_count(const LoopArgs &S, uint64_t seq, int L) {
    __threadfence_system();
    const uint32_t k = (uint32_t)LG_IDX(seq % (uint64_t)S.ring, S.ring, kChkRing);
    if (atomicAdd(&S.done[k], 1u) + 1u == (uint32_t)L) {
        S.done[k] = 0u;  // the slot's next request counts from 0
        __threadfence_system();
        st_release_sys_u64(&S.flags[k], seq + 1);
    }
}

// One persistent launch serving every admitted request of one kind (restarts,
// passes, outputs, atom and torsion maxima): CTAs claim ligands in admission
// order, prepare and dock each one (the batched kernel's docking code, one
// ligand per CTA) as a slot of the arenas named in A0 (ligands and outputs)
// against its request's pocket from the table in S -- all kernel parameters,
// so the docking code reads them as constants -- and the CTA that finishes a
// request's last ligand raises its completion flag.  Waits are bounded: a CTA
// with no ligand to claim for idle_ns leaves; a stop request makes every CTA
// leave after its current ligand; the last CTA out records how the launch
// ended.
template <bool kRank, bool kRigid, int LPR>
__global__ void __launch_bounds__(32 * Rt<LPR>::max_warps, 4 * LG_RT_MIN_BLOCKS / Rt<LPR>::max_warps)
    k_serve_loop(const __grid_constant__ DockArgs A0, const __grid_constant__ LoopArgs S) {
    extern __shared__ __align__(16) char sm[];
    __shared__ long long s_item;
    __shared__ uint64_t s_seq, s_first;
    __shared__ int s_L, s_slot, s_pocket;
    // thread 0's claim state, kept in shared memory so that nothing extra is
    // live in registers while the CTA docks
    __shared__ uint64_t s_hint, s_deadline;
    __shared__ long long s_held;
    __shared__ int s_hk;   // next slot of the held array this CTA drains
    __shared__ int s_why;  // 1 stopped, 2 idle limit, 3 bad item
    if (threadIdx.x == 0) {
        atomicAdd(&S.ctl->live, 1u);
        s_held = -1;
        s_hk = blockIdx.x;
        s_hint = S.first_seq;
        s_deadline = global_ns() + S.idle_ns;
        s_why = 0;
        s_seq = kDescBusy;
        s_first = 0;
        s_L = 0;
    }
    __syncthreads();
    for (;;) {
        if (threadIdx.x == 0) {
            long long held = s_held;
            int hk = s_hk;
            uint64_t deadline = s_deadline, hint = s_hint;
            long long item = loop_claim(S, held, hk, deadline);
            if (item >= 0 && !(s_seq != kDescBusy && (uint64_t)item >= s_first &&
                               (uint64_t)item < s_first + (uint64_t)s_L)) {
                uint64_t sq, f;
                int n, sl, pk;
                if (loop_find(S, item, hint, sq, f, n, sl, pk)) {
                    s_seq = sq;
                    s_first = f;
                    s_L = n;
                    s_slot = sl;
                    s_pocket = pk;
                } else {
                    atomicAdd(&S.ctl->bad, 1u);
                    item = -3;
                }
            }
            s_held = held;
            s_hk = hk;
            s_deadline = deadline;
            s_hint = hint;
            s_why = item >= 0 ? 0 : (int)(-item);
            s_item = item;
        }
        __syncthreads();
        const long long item = s_item;
        if (item < 0) break;
        const int l = s_slot + (int)((uint64_t)item - s_first);
        const int p = s_pocket;
        prep_cta(A0, A0.batch, A0.out, l, (size_t)blockIdx.x, sm);
        LigSrc q;
        q.batch = A0.batch;
        q.dc2g = S.dc2g[p];
        q.thr2g = S.thr2g[p];
        q.rigid_shift_g = S.rigid_shift_g[p];
        dock_ligand_rt<kRank, kRigid, false, LPR>(A0, S.pk[p], A0.out, q, l, sm);
        __syncthreads();
        if (threadIdx.x == 0) loop_count(S, s_seq, s_L);
    }
    if (threadIdx.x == 0) {
        S.held[blockIdx.x] = s_held;  // drained at the CTA's first claim, so free
        if (s_why == 2) atomicAdd(&S.ctl->idle_exits, 1u);
        __threadfence();
        if (atomicSub(&S.ctl->live, 1u) == 1u) {  // the last CTA out
            const int st = ld_acquire_u32(&S.ctl->bad) ? LG_EINVAL
                           : (ld_acquire_u32(&S.ctl->idle_exits) && !ld_acquire_u32(&S.ctl->stop)) ? LG_ETIMEOUT
                                                                                                   : LG_OK;
            S.ctl->status = st;
        }
    }
}

// ================================================================== pocket packing
// Trilinear coefficients of every node's cell, the layout the lookups read
// (Sec. 3.2: the grids stay on the GPU): for node (i, j, k) the 8
// coefficients of the polynomial through the cell's corners, corner indices
// clamped to the last layer, as differences of the FP32 grid values in FP64
// rounded to FP32 -- the overlap grid into cell_o (8 floats per node), the
// vdW and electrostatic grids side by side into cell_ve (16 floats per node).
// Additions only, in one fixed order, so the result is the same on any
// IEEE machine.
__device__ __forceinline__ void pack_one(const float *g, int n, int i, int j, int k, float4 &lo, float4 &hi) {
    const int i1 = min(i + 1, n - 1), j1 = min(j + 1, n - 1), k1 = min(k + 1, n - 1);
    auto at = [&](int a, int b, int c) { return (double)g[((size_t)c * n + b) * n + a]; };
    const double v000 = at(i, j, k), v100 = at(i1, j, k), v010 = at(i, j1, k), v110 = at(i1, j1, k);
    const double v001 = at(i, j, k1), v101 = at(i1, j, k1), v011 = at(i, j1, k1), v111 = at(i1, j1, k1);
    lo = make_float4((float)v000, (float)(v100 - v000), (float)(v010 - v000), (float)(v001 - v000));
    hi = make_float4((float)(v110 - v100 - v010 + v000), (float)(v101 - v100 - v001 + v000),
                     (float)(v011 - v010 - v001 + v000),
                     (float)(v111 - v110 - v101 - v011 + v100 + v010 + v001 - v000));
}

__global__ void k_pack_cells(const float *go, const float *gv, const float *ge, int n, float4 *cell_o, float4 *cell_ve) {
    const size_t n3 = (size_t)n * n * n;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n3; t += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(t % n), j = (int)((t / n) % n), k = (int)(t / ((size_t)n * n));
        float4 lo, hi;
        pack_one(go, n, i, j, k, lo, hi);
        cell_o[2 * t] = lo;
        cell_o[2 * t + 1] = hi;
        pack_one(gv, n, i, j, k, lo, hi);
        cell_ve[4 * t] = lo;
        cell_ve[4 * t + 1] = hi;
        pack_one(ge, n, i, j, k, lo, hi);
        cell_ve[4 * t + 2] = lo;
        cell_ve[4 * t + 3] = hi;
    }
}

cudaError_t launch_pack_cells(const float *go, const float *gv, const float *ge, int n, float4 *cell_o, float4 *cell_ve,
                              int num_sms, cudaStream_t s) {
    const size_t n3 = (size_t)n * n * n;
    const int blocks = (int)std::min<size_t>((n3 + 255) / 256, (size_t)num_sms * 8);
    k_pack_cells<<<blocks, 256, 0, s>>>(go, gv, ge, n, cell_o, cell_ve);
    return cudaGetLastError();
}

// ================================================================== FP32 peak
// FP32 FMA throughput of the device, for the roofline's denominator: every
// thread runs 8 independent FMA chains (enough to cover the pipe's latency
// at 8 warps per SM) for `iters` steps; each FMA is 2 FLOP.  The sums are
// stored so that nothing is dropped.
__global__ void __launch_bounds__(256) k_fp32_peak(float *out, int iters, float a, float b) {
    float x[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = (float)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < 8; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

cudaError_t launch_fp32_peak(float *out, int blocks, int iters, cudaStream_t s) {
    k_fp32_peak<<<blocks, 256, 0, s>>>(out, iters, 0.999999f, 1e-6f);
    return cudaGetLastError();
}

// ================================================================== pose scoring and diagnostics
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

// ================================================================== host side
static size_t al256(size_t v) { return (v + 255) & ~(size_t)255; }

size_t scratch_bytes(int L, int rmax, int rank_slots, int S, int P, int nmax) {
    rmax = rmax > 0 ? rmax : 1;
    size_t b = al256(4 * kHistInts) + 2 * al256(4 * (size_t)L) + al256(24 * (size_t)L) +
               al256(2 * (size_t)L * rmax);
    if (rank_slots > 0) {
        const size_t nm = (size_t)((nmax + 3) & ~3);
        b += al256(12 * (size_t)rank_slots * S * nm) + al256(8 * (size_t)rank_slots * S) +
             al256((size_t)rank_slots * S * P * rmax + 1) + al256(4 * (size_t)rank_slots * S) +
             al256(12 * (size_t)rank_slots * S);
    }
    return b;
}

Scratch carve_scratch(void *base, int L, int rmax, int rank_slots, int S, int P, int nmax) {
    rmax = rmax > 0 ? rmax : 1;
    char *p = (char *)base;
    Scratch s;
    s.hist = (int32_t *)p;
    p += al256(4 * kHistInts);
    s.keys = (int32_t *)p;
    p += al256(4 * (size_t)L);
    s.order = (int32_t *)p;
    p += al256(4 * (size_t)L);
    s.centroid = (double *)p;
    p += al256(24 * (size_t)L);
    s.rot_end = (int16_t *)p;
    p += al256(2 * (size_t)L * rmax);
    s.rk_pose = nullptr;
    s.rk_E = nullptr;
    s.rk_tors = nullptr;
    s.rk_G = nullptr;
    s.rk_cen = nullptr;
    s.rk_slots = rank_slots > 0 ? rank_slots : 0;
    s.rk_floats = 0;
    s.per_cta = 0;
    if (rank_slots > 0) {
        const size_t nm = (size_t)((nmax + 3) & ~3);
        s.rk_floats = 3 * (size_t)rank_slots * S * nm;
        s.rk_pose = (float *)p;
        p += al256(12 * (size_t)rank_slots * S * nm);
        s.rk_E = (double *)p;
        p += al256(8 * (size_t)rank_slots * S);
        s.rk_tors = (uint8_t *)p;
        p += al256((size_t)rank_slots * S * P * rmax + 1);
        s.rk_G = (float *)p;
        p += al256(4 * (size_t)rank_slots * S);
        s.rk_cen = (float *)p;
    }
    return s;
}

template <typename K>
static cudaError_t kernel_attributes(K kernel, int W, int smem, int *ctas_per_sm) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, kernel, 32 * W, smem);
}

// The batched kernel of a feature set and restart tile, called with the
// launch's arguments.  Tiles other than 4 lanes per restart exist for the
// forms without ranking and decision ranks (cudaErrorInvalidValue otherwise).
template <typename F>
static cudaError_t with_batched(bool ranking, bool rigid, bool trace, int lanes, F &&f) {
    if (lanes != 4) {
        if (ranking || trace) return cudaErrorInvalidValue;
        switch (lanes) {
        case 2: return rigid ? f(k_dock_batched<false, true, false, 2>) : f(k_dock_batched<false, false, false, 2>);
        case 8: return rigid ? f(k_dock_batched<false, true, false, 8>) : f(k_dock_batched<false, false, false, 8>);
        case 16: return rigid ? f(k_dock_batched<false, true, false, 16>) : f(k_dock_batched<false, false, false, 16>);
        default: return cudaErrorInvalidValue;
        }
    }
    if (ranking) {
        if (rigid) return trace ? f(k_dock_batched<true, true, true, 4>) : f(k_dock_batched<true, true, false, 4>);
        return trace ? f(k_dock_batched<true, false, true, 4>) : f(k_dock_batched<true, false, false, 4>);
    }
    if (rigid) return trace ? f(k_dock_batched<false, true, true, 4>) : f(k_dock_batched<false, true, false, 4>);
    return trace ? f(k_dock_batched<false, false, true, 4>) : f(k_dock_batched<false, false, false, 4>);
}

cudaError_t dock_kernel_attributes(int W, int smem, int *ctas_per_sm, bool ranking, bool rigid, bool trace, int lanes) {
    return with_batched(ranking, rigid, trace, lanes,
                        [&](auto kernel) { return kernel_attributes(kernel, W, smem, ctas_per_sm); });
}

cudaError_t multi_kernel_attributes(int W, int smem, int *ctas_per_sm, bool ranking, bool rigid) {
    if (ranking)
        return rigid ? kernel_attributes(k_dock_multi<true, true>, W, smem, ctas_per_sm)
                     : kernel_attributes(k_dock_multi<true, false>, W, smem, ctas_per_sm);
    return rigid ? kernel_attributes(k_dock_multi<false, true>, W, smem, ctas_per_sm)
                 : kernel_attributes(k_dock_multi<false, false>, W, smem, ctas_per_sm);
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
        k_sort_scan<<<1, 32, 0, s>>>(a.scr.hist, L);
        k_sort_scatter<<<blocks, 256, 0, s>>>(L, a.scr.keys, a.scr.hist, a.scr.order);
        *launches += 2;
    }
    return cudaGetLastError();
}

cudaError_t launch_dock_plain(const DockArgs &a, int ligand, int slot, cudaStream_t s) {
    const int smem = a.ranking ? (a.ly.total > a.ly.cta_bytes + rank_smem_bytes(a.S) ? a.ly.total
                                                                                    : a.ly.cta_bytes + rank_smem_bytes(a.S))
                               : a.ly.total;
    k_dock_plain<<<1, 32 * a.ly.W, smem, s>>>(a, ligand, slot);
    return cudaGetLastError();
}

// Launch configuration of a docking launch; with a.l2_bytes > 0 it carries the
// pocket's L2 access-policy window (overlap-grid cells marked persisting in
// the context's persisting L2 set-aside, other traffic streaming).
struct DockLaunch {
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr[1];
    DockLaunch(const DockArgs &a, int grid, int smem, cudaStream_t s) {
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(32 * a.ly.W);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        if (a.l2_bytes > 0) {
            attr[0].id = cudaLaunchAttributeAccessPolicyWindow;
            attr[0].val.accessPolicyWindow.base_ptr = const_cast<void *>(a.l2_base);
            attr[0].val.accessPolicyWindow.num_bytes = a.l2_bytes;
            attr[0].val.accessPolicyWindow.hitRatio = a.l2_hit;
            attr[0].val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
            attr[0].val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
        }
    }
};

cudaError_t launch_dock_batched(const DockArgs &a, int grid, int smem, cudaStream_t s) {
    DockLaunch dl(a, grid, smem, s);
    return with_batched(a.ranking, a.rigid_steps > 0, a.out.decision_rank != nullptr, a.lanes,
                        [&](auto kernel) { return cudaLaunchKernelEx(&dl.cfg, kernel, a); });
}

cudaError_t launch_dock_multi(const DockArgs &a, const MultiDev &m, int grid, int smem, cudaStream_t s) {
    DockLaunch dl(a, grid, smem, s);
    const bool rigid = a.rigid_steps > 0;
    if (a.ranking && rigid) return cudaLaunchKernelEx(&dl.cfg, k_dock_multi<true, true>, a, m);
    if (a.ranking) return cudaLaunchKernelEx(&dl.cfg, k_dock_multi<true, false>, a, m);
    if (rigid) return cudaLaunchKernelEx(&dl.cfg, k_dock_multi<false, true>, a, m);
    return cudaLaunchKernelEx(&dl.cfg, k_dock_multi<false, false>, a, m);
}

// The serving loop of a feature set and restart tile (16 lanes per restart
// without ranking only; cudaErrorInvalidValue for other tiles).
template <typename F>
static cudaError_t with_loop(bool ranking, bool rigid, int lanes, F &&f) {
    if (lanes == 16 && !ranking) return rigid ? f(k_serve_loop<false, true, 16>) : f(k_serve_loop<false, false, 16>);
    if (lanes != 4) return cudaErrorInvalidValue;
    if (ranking) return rigid ? f(k_serve_loop<true, true, 4>) : f(k_serve_loop<true, false, 4>);
    return rigid ? f(k_serve_loop<false, true, 4>) : f(k_serve_loop<false, false, 4>);
}

cudaError_t loop_kernel_attributes(int W, int smem, int *ctas_per_sm, bool ranking, bool rigid, int lanes) {
    return with_loop(ranking, rigid, lanes,
                     [&](auto kernel) { return kernel_attributes(kernel, W, smem, ctas_per_sm); });
}

cudaError_t launch_serve_loop(const DockArgs &a, const LoopArgs &la, int grid, int smem, cudaStream_t s) {
    return with_loop(a.ranking, a.rigid_steps > 0, a.lanes, [&](auto kernel) {
        kernel<<<grid, 32 * a.ly.W, smem, s>>>(a, la);
        return cudaGetLastError();
    });
}

cudaError_t launch_flatten(const FlatArgs &f, int L, cudaStream_t s) {
    const int smem = kFlatWarps * flat_warp_bytes(f.nmax);
    cudaError_t e = cudaFuncSetAttribute(k_flatten, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    k_flatten<<<(L + kFlatWarps - 1) / kFlatWarps, 32 * kFlatWarps, smem, s>>>(f);
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
