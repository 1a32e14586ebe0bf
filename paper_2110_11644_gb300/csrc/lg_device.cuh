// Device arithmetic shared by the docking kernels (lg_kernels.cu).
//
// Every floating-point step of the docking method is written once here, with
// explicit fmaf / products, so the two kernel forms (plain: one warp per
// restart; batched: restart-tiled warps) perform the same operations in the
// same order and produce bit-identical results.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lg_internal.h"

namespace lg {

#define LG_FULL 0xffffffffu

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

// Rigid pose of restart r: rotation (row-major) from Shoemake's uniform
// quaternion of three 24-bit uniforms, and the pocket-point index.
struct Pose {
    float R[9];
    uint32_t pp;
};

__device__ __forceinline__ Pose restart_pose(uint64_t uid, uint32_t r, uint2 key, int n_pp) {
    const uint4 x4 = philox4x32_10(make_uint4((uint32_t)uid, (uint32_t)(uid >> 32), r, 0u), key);
    const float u0 = (float)(x4.x >> 8) * 5.9604644775390625e-08f;  // 2^-24
    const float u1 = (float)(x4.y >> 8) * 5.9604644775390625e-08f;
    const float u2 = (float)(x4.z >> 8) * 5.9604644775390625e-08f;
    const float s1 = sqrtf(1.0f - u0), s2 = sqrtf(u0);
    float sn1, cs1, sn2, cs2;
    sincospif(2.0f * u1, &sn1, &cs1);
    sincospif(2.0f * u2, &sn2, &cs2);
    const float qx = s1 * sn1, qy = s1 * cs1, qz = s2 * sn2, qw = s2 * cs2;
    Pose P;
    P.R[0] = 1.0f - 2.0f * (qy * qy + qz * qz);
    P.R[1] = 2.0f * (qx * qy - qw * qz);
    P.R[2] = 2.0f * (qx * qz + qw * qy);
    P.R[3] = 2.0f * (qx * qy + qw * qz);
    P.R[4] = 1.0f - 2.0f * (qx * qx + qz * qz);
    P.R[5] = 2.0f * (qy * qz - qw * qx);
    P.R[6] = 2.0f * (qx * qz - qw * qy);
    P.R[7] = 2.0f * (qy * qz + qw * qx);
    P.R[8] = 1.0f - 2.0f * (qx * qx + qy * qy);
    P.pp = (uint32_t)(((uint64_t)(x4.w >> 8) * (uint64_t)n_pp) >> 24);
    return P;
}

// R v + t
__device__ __forceinline__ float3 rot_add(const float *R, float vx, float vy, float vz, float tx, float ty, float tz) {
    return make_float3(fmaf(R[0], vx, fmaf(R[1], vy, fmaf(R[2], vz, tx))),
                       fmaf(R[3], vx, fmaf(R[4], vy, fmaf(R[5], vz, ty))),
                       fmaf(R[6], vx, fmaf(R[7], vy, fmaf(R[8], vz, tz))));
}

// R v
__device__ __forceinline__ float3 rot_vec(const float *R, float vx, float vy, float vz) {
    return make_float3(fmaf(R[0], vx, fmaf(R[1], vy, R[2] * vz)), fmaf(R[3], vx, fmaf(R[4], vy, R[5] * vz)),
                       fmaf(R[6], vx, fmaf(R[7], vy, R[8] * vz)));
}

// ------------------------------------------------------------------ bounds checks
// A debug build (-DLG_CHECKS) checks the computed indices of grid cells,
// shared-memory lists and scratch slots: an index outside [0, bound) is
// counted, the first one recorded (site, index, bound), and the access goes to
// the nearest in-range element instead, so it stays in bounds; the host turns
// a record into an error of the call.  Other builds compile the checks away.
enum CheckSite {
    kChkCell = 1,      // overlap-grid cell of a torsion-step lookup
    kChkCellVE,        // potential-grid cell of a pose score
    kChkNear,          // near-atom list entry
    kChkPool,          // clash-pair pool entry
    kChkDecision,      // decision record of a restart slot
    kChkRankSlot,      // ranking scratch slot
    kChkAtom,          // atom index of a moving or fixed atom
    kChkRing,          // request-descriptor slot of the serving loop
};
#ifdef LG_CHECKS
__device__ int lg_check_rec[4];  // site, index, bound of the first failure; failures
__device__ __forceinline__ long long lg_checked(long long idx, long long bound, int site) {
    if (idx >= 0 && idx < bound) return idx;
    if (atomicAdd(&lg_check_rec[3], 1) == 0) {
        lg_check_rec[0] = site;
        lg_check_rec[1] = (int)idx;
        lg_check_rec[2] = (int)bound;
    }
    return idx < 0 ? 0 : bound - 1;
}
#define LG_IDX(idx, bound, site) lg_checked((long long)(idx), (long long)(bound), (site))
#else
#define LG_IDX(idx, bound, site) (idx)
#endif

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

struct GridK {  // lookup constants of one packed grid
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

// One 32-byte cell (8 coefficients) with a single 256-bit read-only load
// (sm_100+); cells are 32-byte aligned.
// Cells are rarely reused from L1 (scattered lookups), so they bypass L1
// allocation; this measured faster than caching them.
#ifndef LG_CELL_LOAD
#define LG_CELL_LOAD "ld.global.nc.L1::no_allocate.v8.f32"
#endif
__device__ __forceinline__ void load_cell(const float4 *p, float4 &lo, float4 &hi) {
    asm(LG_CELL_LOAD " {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(lo.x), "=f"(lo.y), "=f"(lo.z), "=f"(lo.w), "=f"(hi.x), "=f"(hi.y), "=f"(hi.z), "=f"(hi.w)
                 : "l"(p));
}

// Overlap-field value at an index-space point known to lie in [0, n-1]^3.
__device__ __forceinline__ float lookup_in(const GridK &G, float gx, float gy, float gz) {
    float tx, ty, tz;
    const float fx = floor_frac(gx, tx), fy = floor_frac(gy, ty), fz = floor_frac(gz, tz);
    float4 lo, hi;
    load_cell(G.cells + 2 * (size_t)LG_IDX(cell_index(tx, ty, tz, G.n, G.n2, G.moff), (size_t)G.n2 * G.n, kChkCell),
              lo, hi);
    return cell_eval(lo, hi, fx, fy, fz);
}

// Overlap-field value at any index-space point (clamped to the box; equal to
// lookup_in for points inside the box).
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
    const float4 *p =
        G.cells + 4 * (size_t)LG_IDX(cell_index(tx, ty, tz, G.n, G.n2, G.moff), (size_t)G.n2 * G.n, kChkCellVE);
    float4 vlo, vhi, elo, ehi;
    load_cell(p, vlo, vhi);
    load_cell(p + 2, elo, ehi);
    const float v = cell_eval(vlo, vhi, fx, fy, fz);
    const float e = cell_eval(elo, ehi, fx, fy, fz);
    return fmaf(w, v, fmaf(q, e, P.k_out * out));
}

// ------------------------------------------------------------------ torsion geometry
// Unit axis of a bond vector.
__device__ __forceinline__ float3 unit_axis(float4 v) {
    const float inv = rnorm3df(v.x, v.y, v.z);
    return make_float3(v.x * inv, v.y * inv, v.z * inv);
}

// The circle a moving atom x traces about the axis u through xb:
//   x(theta) = p + e1 cos(theta) + e2 sin(theta),
// p its centre (P = p + c0 in index space), e1 = radius vector at theta = 0,
// e2 = u x (x - xb), r2 = |e1|^2; `inside` when the whole circle lies in the
// grid box with a margin.
struct Circle {
    float Px, Py, Pz;
    float e1x, e1y, e1z;
    float e2x, e2y, e2z;
    float r2;
    float px, py, pz;
    bool inside;
};

__device__ __forceinline__ Circle make_circle(float xi, float yi, float zi, float xbx, float xby, float xbz, float3 u,
                                              float c0, float gmax) {
    Circle C;
    const float dx = xi - xbx, dy = yi - xby, dz = zi - xbz;
    const float w = fmaf(u.x, dx, fmaf(u.y, dy, u.z * dz));
    C.px = fmaf(w, u.x, xbx);
    C.py = fmaf(w, u.y, xby);
    C.pz = fmaf(w, u.z, xbz);
    C.e1x = fmaf(-w, u.x, dx);
    C.e1y = fmaf(-w, u.y, dy);
    C.e1z = fmaf(-w, u.z, dz);
    C.e2x = fmaf(u.y, dz, -u.z * dy);
    C.e2y = fmaf(u.z, dx, -u.x * dz);
    C.e2z = fmaf(u.x, dy, -u.y * dx);
    C.Px = C.px + c0;
    C.Py = C.py + c0;
    C.Pz = C.pz + c0;
    C.r2 = fmaf(C.e1x, C.e1x, fmaf(C.e1y, C.e1y, C.e1z * C.e1z));
    const float rx = fabsf(C.e1x) + fabsf(C.e2x), ry = fabsf(C.e1y) + fabsf(C.e2y), rz = fabsf(C.e1z) + fabsf(C.e2z);
    const float lim = gmax - 1e-3f;
    C.inside = C.Px - rx >= 1e-3f && C.Px + rx <= lim && C.Py - ry >= 1e-3f && C.Py + ry <= lim &&
               C.Pz - rz >= 1e-3f && C.Pz + rz <= lim;
    return C;
}

// Index-space point of a circle at a step with cosine c and sine s.
__device__ __forceinline__ float3 circle_index(float Px, float Py, float Pz, float e1x, float e1y, float e1z, float e2x,
                                               float e2y, float e2z, float c, float s) {
    return make_float3(fmaf(e2x, s, fmaf(e1x, c, Px)), fmaf(e2y, s, fmaf(e1y, c, Py)), fmaf(e2z, s, fmaf(e1z, c, Pz)));
}

// Clash coefficients of a moving atom's circle against a fixed atom j:
//   |x(theta) - x_j|^2 = C + A2 cos(theta) + B2 sin(theta).
// `near` is false only when the minimum over the circle, C - sqrt(A2^2 + B2^2),
// is certainly >= dc2 (the test keeps a 1e-4 relative margin, so rounding can
// never drop a pair that clashes at some step).
struct PairC {
    float C, A2, B2;
    bool near;
};

__device__ __forceinline__ PairC pair_coeffs(float px, float py, float pz, float e1x, float e1y, float e1z, float e2x,
                                             float e2y, float e2z, float r2, float xj, float yj, float zj, float dc2) {
    PairC q;
    const float wx = px - xj, wy = py - yj, wz = pz - zj;
    const float aa = fmaf(wx, e1x, fmaf(wy, e1y, wz * e1z));
    const float bb = fmaf(wx, e2x, fmaf(wy, e2y, wz * e2z));
    q.C = fmaf(wx, wx, fmaf(wy, wy, fmaf(wz, wz, r2)));
    const float T = q.C - dc2;
    const float s2 = fmaf(aa, aa, bb * bb);
    q.near = T <= 0.0f || T * T < 4.0004f * s2;
    q.A2 = 2.0f * aa;
    q.B2 = 2.0f * bb;
    return q;
}

__device__ __forceinline__ bool pair_clash(float C, float A2, float B2, float c, float s, float dc2) {
    return fmaf(B2, s, fmaf(A2, c, C)) < dc2;
}

// Rotate a point about the axis u through xb by (c, s) (same circle form).
__device__ __forceinline__ float3 rotate_point(float x, float y, float z, float xbx, float xby, float xbz, float3 u,
                                               float c, float s) {
    const float dx = x - xbx, dy = y - xby, dz = z - xbz;
    const float w = fmaf(u.x, dx, fmaf(u.y, dy, u.z * dz));
    const float e1x = fmaf(-w, u.x, dx), e1y = fmaf(-w, u.y, dy), e1z = fmaf(-w, u.z, dz);
    const float e2x = fmaf(u.y, dz, -u.z * dy), e2y = fmaf(u.z, dx, -u.x * dz), e2z = fmaf(u.x, dy, -u.y * dx);
    return make_float3(fmaf(e2x, s, fmaf(e1x, c, fmaf(w, u.x, xbx))), fmaf(e2y, s, fmaf(e1y, c, fmaf(w, u.y, xby))),
                       fmaf(e2z, s, fmaf(e1z, c, fmaf(w, u.z, xbz))));
}

// Rigid moves of the whole ligand: candidate 0 stays; 1..6 shift by +d, -d
// along x, y, z; 7..12 turn by +a, -a about the x, y, z axes through the
// centroid (cx, cy, cz) (right-hand rule; (ca, sa) = (cos a, sin a)).
constexpr int kRigidCandidates = 13;

__device__ __forceinline__ float3 rigid_candidate(int cand, float x, float y, float z, float cx, float cy, float cz,
                                                  float d, float ca, float sa) {
    float3 r = make_float3(x, y, z);
    if (cand >= 1 && cand <= 6) {
        const float dd = (cand & 1) ? d : -d;
        if (cand <= 2) r.x += dd;
        else if (cand <= 4) r.y += dd;
        else r.z += dd;
    } else if (cand >= 7) {
        const float s = (cand & 1) ? sa : -sa;
        if (cand <= 8) {         // about x: (y, z)
            const float vj = y - cy, vk = z - cz;
            r.y = cy + fmaf(ca, vj, -s * vk);
            r.z = cz + fmaf(s, vj, ca * vk);
        } else if (cand <= 10) { // about y: (z, x)
            const float vj = z - cz, vk = x - cx;
            r.z = cz + fmaf(ca, vj, -s * vk);
            r.x = cx + fmaf(s, vj, ca * vk);
        } else {                 // about z: (x, y)
            const float vj = x - cx, vk = y - cy;
            r.x = cx + fmaf(ca, vj, -s * vk);
            r.y = cy + fmaf(s, vj, ca * vk);
        }
    }
    return r;
}

// A direction under candidate `cand` (turns only; shifts leave it unchanged).
__device__ __forceinline__ float4 rigid_candidate_vec(int cand, float4 v, float ca, float sa) {
    if (cand < 7) return v;
    const float3 r = rigid_candidate(cand, v.x, v.y, v.z, 0.0f, 0.0f, 0.0f, 0.0f, ca, sa);
    return make_float4(r.x, r.y, r.z, v.w);
}

// Rotate a vector about the unit axis u by (c, s) (Rodrigues).
__device__ __forceinline__ float4 rotate_vec(float4 v, float3 u, float c, float s) {
    const float uv = fmaf(u.x, v.x, fmaf(u.y, v.y, u.z * v.z));
    const float cx = fmaf(u.y, v.z, -u.z * v.y), cy = fmaf(u.z, v.x, -u.x * v.z), cz = fmaf(u.x, v.y, -u.y * v.x);
    const float k1 = uv * (1.0f - c);
    return make_float4(fmaf(cx, s, fmaf(v.x, c, k1 * u.x)), fmaf(cy, s, fmaf(v.y, c, k1 * u.y)),
                       fmaf(cz, s, fmaf(v.z, c, k1 * u.z)), 0.0f);
}

// Better of two (score, step) candidates: higher score, lower step on ties.
__device__ __forceinline__ bool better(float s1, int t1, float s0, int t0) { return s1 > s0 || (s1 == s0 && t1 < t0); }

}  // namespace lg
