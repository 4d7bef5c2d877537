// k_push.cu -- fused field gather, Boris push, move and Esirkepov current
// deposition for the mixed (int32 cell + FP32 offset) particle form.
//
// One CTA works on one supercell at a time (Sec. 2.1: a supercell maps to a
// block, its threads share the supercell's particles); CTAs are persistent
// and pull supercells from a work counter (one item ahead), so boxes of any
// size and occupancy share one launch.  Per supercell:
//   1. stage the E and B tile (supercell + G guard cells below, G = 1 for
//      CIC/TSC, 2 with PCS) from HBM into shared memory with 16-byte
//      asynchronous copies;
//   2. zero a shared J tile of the same extent;
//   3. every thread takes particles of the supercell's frame lists: gather
//      E, B from shared memory (CIC 2x2x2 / TSC 3x3x3 / PCS 4x4x4 weights
//      per component at its Yee position, Sec. 4; optionally one order lower
//      along the component's staggered axes, the energy-conserving variant),
//      relativistic Boris push, move, then Esirkepov deposition (Sec. 4) into
//      the shared J tile with shared atomics; the particles that stay go back
//      to the list compacted (in chunk order, so the leavers' slots close up
//      as the list is written); particles that leave the supercell collect in
//      a shared leaver buffer that the CTA hands to the move buffer at its
//      next work item (or leave through a subdomain slab's z face into a
//      migrant message, or through a y face of an open-y box out of the
//      simulation);
//   4. add the J tile to the guard-padded global J with 16-byte vector
//      atomics (neighbouring supercells overlap in their guard cells).
//
// Esirkepov (2001): with 1D shape factors S0 (old) and S1 (new) on a common
// window and DS = S1 - S0, the x current on the half node i+1/2 is
//   Jx(i+1/2, j, k) = -(q w hx / (V dt)) * sum_{i' <= i} DSx(i')
//                     * [S0y S0z + DSy S0z / 2 + S0y DSz / 2 + DSy DSz / 3](j, k)
// i.e. an outer product of a prefix sum along x and a transverse factor.
//
// Particles go through a chunk of at most 256 at a time in the order of a
// counting sort by nearest node (cell for CIC and PCS), so the lanes of a
// warp read neighbouring field words (shared-memory broadcasts).  Every
// sort_every-th step (a sort pass) stages each chunk in shared memory, sorts
// it and writes it back to the list in sorted order; the steps between push
// the lists in stored order from the chunk stage, which an asynchronous copy
// fills while the previous chunk deposits.  The push writes a deposit record
// per particle; the deposit then runs in a lane order whose neighbours are
// kDepStride sorted positions apart, so one warp's atomics land on different
// nodes.  The current of a chunk accumulates in fixed point (see
// chunk_scale).  Two deposit paths, both exact forms of that formula:
//   common: on every axis the move stays on one spline piece -- the old and
//     the new position round to the same node (TSC) / stay in the same cell
//     (CIC, PCS) -- so the union of the two supports is 3 (TSC) / 2 (CIC) /
//     4 (PCS) nodes and DS has closed per-node forms in the displacement D
//     (no cancellation in FP32); 54 (TSC) / 12 (CIC) / 144 (PCS) shared
//     atomics, no branches;
//   general: the rest (a few percent of particles) are listed and deposited
//     on a 4-node (CIC, TSC) or 5-node (PCS) window: set aside (up to
//     kGenDefer per list) and deposited lane-parallel after the list's last
//     chunk with their own fixed-point scale; beyond that, with their chunk:
//     whole groups of 32 lane-parallel, the leftover moves one per warp with
//     all 32 lanes on the move's current lines.
// The shared tiles use a row pitch of 4 mod 8 floats, so that rows are
// 16-byte aligned (the E/B tile arrives by cp.async, the J tile leaves as
// float4) and the 32 banks spread over neighbouring rows.
#include "pic_internal.cuh"
#include "tma.cuh"

#include <cmath>

namespace pic {

// General-window moves of a frame list deposited together after its last
// chunk (more are deposited with their own chunk).
constexpr int kGenDefer = 64;
// Particles changing supercell that a CTA collects in shared memory and hands
// to the move buffer at the start of its next work item (more go straight
// to the move buffer).
constexpr int kLeaverBuf = 48;
// Lane stride of the deposit over the node-sorted chunk: 4 spreads one
// warp's 54 atomics per particle over the banks better than 1 (neighbours
// share a node) or C / 32 (random over the tile).
constexpr int kDepStride = 4;

// G = guard cells below the supercell (the fields' global guards match):
// 1 for CIC/TSC, 2 when a PCS species is present (its support reaches two
// nodes below the cell and, for a move across a cell face, three above).
template <int LX_, int LY_, int LZ_, int G_ = 1>
struct Tile {
    static constexpr int LX = LX_, LY = LY_, LZ = LZ_, G = G_;
    static constexpr int GO = G - 1;  // tile index of node l - 1 is l + GO
    // x: G below, 3 (CIC/TSC) / 6 (PCS) above, 16-byte rows; y, z: G below, 2 / 3 above
    static constexpr int TX = G == 1 ? LX + 4 : LX + 8;
    static constexpr int TY = G == 1 ? LY + 3 : LY + 5;
    static constexpr int TZ = G == 1 ? LZ + 3 : LZ + 5;
    // shared-memory row pitch: the first multiple of 4 at or above TX that is
    // 4 mod 8, so that rows are 16-byte aligned and consecutive rows start 12
    // (or 20) banks apart
    static constexpr int PX = (TX % 8 == 4) ? TX : (TX % 8 == 0 ? TX + 4 : ((TX + 3) / 4) * 4);
    static constexpr int N = PX * TY * TZ;  // shared floats per component
    static constexpr int S = LX * LY * LZ;
    // the B tile starts here (floats from the E tile's start): 128-byte
    // aligned, like the E tile, for its tensor load
    static constexpr int BOFF = ((3 * N + 31) / 32) * 32;
    // shared floats of the field tiles and the two current tiles
    static constexpr int TILES = BOFF + 9 * N;
    static_assert(PX % 4 == 0 && N % 4 == 0, "tile rows and components are 16-byte aligned");
};

// ------------------------------------------------------------ shape factors

// TSC (quadratic spline, Hockney & Eastwood) at distance d, branch-free.
__host__ __device__ __forceinline__ float tsc_S(float d)
{
    float a = fabsf(d);
    float t = fmaxf(1.5f - a, 0.0f);
    return a <= 0.5f ? 0.75f - a * a : 0.5f * t * t;
}

// S(d0 + D) - S(d0) for TSC without ever forming d1 = d0 + D (rounding d1
// costs ~6e-8 absolute, which is a large relative error on a DS of order D
// for slow particles).  On one spline piece the difference is factored
// through D; across a piece boundary p (|d| = 1/2 or 3/2) it is the sum of
// the two pieces' differences to p, with the exact distance d0 -> p
// (Sterbenz) and the remainder D - (p - d0).  The spline is C1 at its joins,
// so a misjudged side of p changes the result only at second order.
__host__ __device__ __forceinline__ float tsc_dS(float d0, float D)
{
    const float a0 = fabsf(d0);
    const float s0 = d0 >= 0.0f ? 1.0f : -1.0f;
    if (a0 <= 0.5f) {
        const float d1 = d0 + D;  // classification only
        if (fabsf(d1) <= 0.5f)
            return -D * (2.0f * d0 + D);                 // centre piece: d0^2 - d1^2
        const float p = d1 >= 0.0f ? 0.5f : -0.5f;
        const float u1 = p - d0;                          // exact distance to the join
        const float t = (d1 >= 0.0f ? 1.0f : -1.0f) * (D - u1);  // |d1| - 1/2 >= 0
        return -u1 * (p + d0) + t * (0.5f * t - 1.0f);   // centre to p, then outer piece
    }
    const float a1 = a0 + s0 * D;  // |d1| on this side (classification)
    if (a0 < 1.5f) {
        if (a1 <= 0.5f) {                                 // outer piece into the centre
            const float p = 0.5f * s0;
            const float t0 = a0 - 0.5f;                   // exact
            const float u2 = s0 * t0 + D;                 // d1 - p
            return t0 * (1.0f - 0.5f * t0) - u2 * (2.0f * p + u2);
        }
        if (a1 < 1.5f)                                    // outer piece
            return -0.5f * s0 * D * (3.0f - 2.0f * a0 - s0 * D);
        const float r0 = 1.5f - a0;                       // out of the support
        return -0.5f * r0 * r0;
    }
    if (a1 < 1.5f) {                                      // into the support
        const float r1 = (1.5f - a0) - s0 * D;            // 1.5 - |d1|
        return 0.5f * r1 * r1;
    }
    return 0.0f;
}

__host__ __device__ __forceinline__ float cic_S(float d) { return fmaxf(0.0f, 1.0f - fabsf(d)); }

// S(d0 + D) - S(d0) for CIC, the same way: across the node (d = 0) the
// difference is s0 (2 d0 + D); across the support edge (|d| = 1, a kink, so
// the side is decided exactly: 1 - |d0| is exact and compared with s0 D)
// it is the distance to the edge.
__host__ __device__ __forceinline__ float cic_dS(float d0, float D)
{
    const float a0 = fabsf(d0);
    const float s0 = d0 >= 0.0f ? 1.0f : -1.0f;
    if (a0 < 1.0f) {
        if (a0 >= 0.5f && s0 * D >= 1.0f - a0)
            return -(1.0f - a0);                          // out of the support
        const float d1 = d0 + D;                          // its sign is exact
        if ((d1 >= 0.0f) == (d0 >= 0.0f))
            return -s0 * D;
        return s0 * (2.0f * d0 + D);                      // across the node
    }
    if (-s0 * D > a0 - 1.0f)
        return (1.0f - a0) - s0 * D;                      // into the support: 1 - |d1|
    return 0.0f;
}

// PCS (cubic B-spline) at distance d.
__host__ __device__ __forceinline__ float pcs_S(float d)
{
    const float a = fabsf(d);
    if (a < 1.0f)
        return (4.0f - 6.0f * a * a + 3.0f * a * a * a) * (1.0f / 6.0f);
    const float t = fmaxf(2.0f - a, 0.0f);
    return t * t * t * (1.0f / 6.0f);
}

// S(d0 + D) - S(d0) on one spline piece (the piece of the segment's midpoint),
// factored through D: central piece (|d| < 1, sign s fixed)
//   D [-(d0 + d1) + s (d0^2 + d0 d1 + d1^2) / 2],
// outer piece (1 <= |d| < 2, a = 2 - s d)   -s D (a0^2 + a0 a1 + a1^2) / 6.
__host__ __device__ __forceinline__ float pcs_seg(float d0, float D)
{
    const float d1 = d0 + D;
    const float m = d0 + 0.5f * D;
    const float s = m >= 0.0f ? 1.0f : -1.0f;
    const float am = fabsf(m);
    if (am < 1.0f)
        return D * (-(d0 + d1) + 0.5f * s * (d0 * d0 + d0 * d1 + d1 * d1));
    if (am < 2.0f) {
        const float a0 = 2.0f - s * d0, a1 = 2.0f - s * d1;
        return -s * D * (a0 * a0 + a0 * a1 + a1 * a1) * (1.0f / 6.0f);
    }
    return 0.0f;
}

// S(d0 + D) - S(d0) for PCS without forming the difference of two values:
// the pieces join at the integers (the spline is C2 there), and a move of
// less than half a cell crosses at most one join p, where the difference is
// split at p with the exact distance p - d0.
__host__ __device__ __forceinline__ float pcs_dS(float d0, float D)
{
    const float d1 = d0 + D;  // classification only
    const float lo = fminf(d0, d1), hi = fmaxf(d0, d1);
    const float p = floorf(hi);
    if (p > lo && fabsf(p) <= 2.0f) {
        const float u = p - d0;
        return pcs_seg(d0, u) + pcs_seg(p, D - u);
    }
    return pcs_seg(d0, D);
}

// Gather weights along one axis for a particle at offset o in [0,1) of its
// cell; the tile coordinate of the particle's cell is l + 1.  "i" = field
// sampled at integer nodes along this axis, "h" = at half nodes.  For the
// integer nodes the weights are also the particle's shape S0 at the nodes
// a-1, a, a+1 (TSC, a = round(o)) or 0, 1 (CIC): the deposit reuses them.
// red: the energy-conserving variant, one order lower at the half nodes
// (CIC inside the TSC window, nearest node inside the CIC window).
// l is the tile index of node (cell - 1): cell + GO.
template <int SHAPE>
struct AxisW {
    static constexpr int NW = SHAPE == 2 ? 3 : (SHAPE == 3 ? 4 : 2);
    int bi, bh;  // tile index of the first node
    float wi[NW], wh[NW];
    __device__ __forceinline__ AxisW(int l, float o, bool red)
    {
        if (SHAPE == 3) {
            // integer nodes cell-1 .. cell+2; half nodes m0 .. m0+3 with
            // m0 = cell - 2 + up (the half node m + 1/2 is stored at index m)
            bi = l;
            wi[0] = pcs_S(o + 1.0f);
            wi[1] = pcs_S(o);
            wi[2] = pcs_S(o - 1.0f);
            wi[3] = pcs_S(o - 2.0f);
            const bool up = o >= 0.5f;
            bh = l - 1 + (up ? 1 : 0);
            if (red) {  // TSC at the half nodes cell-1, cell, cell+1
                const float a = 1.0f - o, c = o, m = 0.75f - (o - 0.5f) * (o - 0.5f);
                wh[0] = up ? 0.5f * a * a : 0.0f;
                wh[1] = up ? m : 0.5f * a * a;
                wh[2] = up ? 0.5f * c * c : m;
                wh[3] = up ? 0.0f : 0.5f * c * c;
            } else {
                const float h = o + (up ? 0.5f : 1.5f);  // distance to half node m0
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    wh[k] = pcs_S(h - (float)k);
            }
        } else if (SHAPE == 2) {
            bool up = o >= 0.5f;
            const float di = up ? o - 1.0f : o;  // offset from the nearest node
            bi = l + (up ? 1 : 0);
            float a = 0.5f - di, c = 0.5f + di;
            wi[0] = 0.5f * a * a;
            wi[1] = 0.75f - di * di;
            wi[2] = 0.5f * c * c;
            float dh = o - 0.5f;
            bh = l;  // half nodes l - 1/2, l + 1/2, l + 3/2
            if (red) {
                wh[0] = up ? 0.0f : 0.5f - o;
                wh[1] = up ? 1.5f - o : 0.5f + o;
                wh[2] = up ? o - 0.5f : 0.0f;
            } else {
                float ah = 0.5f - dh, ch = 0.5f + dh;
                wh[0] = 0.5f * ah * ah;
                wh[1] = 0.75f - dh * dh;
                wh[2] = 0.5f * ch * ch;
            }
        } else {
            bi = l + 1;
            wi[0] = 1.0f - o;
            wi[1] = o;
            bool up = o >= 0.5f;
            float dh = up ? o - 0.5f : o + 0.5f;
            bh = l + (up ? 1 : 0);  // half nodes bh - 1/2 .. : the cell's own is l + 1/2
            wh[0] = red ? (up ? 1.0f : 0.0f) : 1.0f - dh;
            wh[1] = red ? (up ? 0.0f : 1.0f) : dh;
        }
    }
};

template <int NW, int PX, int TY>
__device__ __forceinline__ float gather_comp(const float* __restrict__ F, int bx, int by, int bz,
                                             const float* wx, const float* wy, const float* wz)
{
    float acc = 0.0f;
#pragma unroll
    for (int c = 0; c < NW; ++c) {
#pragma unroll
        for (int b = 0; b < NW; ++b) {
            const float* row = F + ((bz + c) * TY + (by + b)) * PX + bx;
            float r = 0.0f;
#pragma unroll
            for (int a = 0; a < NW; ++a)
                r = fmaf(row[a], wx[a], r);
            acc = fmaf(r, wy[b] * wz[c], acc);
        }
    }
    return acc;
}

// Two components at once on the packed FP32 pipe (two independent FMAs per
// instruction, each rounded as the scalar fmaf: the same result as two
// gather_comp calls).
template <int NW, int PX, int TY>
__device__ __forceinline__ float2 gather_pair(const float* __restrict__ F1, int x1, int y1, int z1,
                                              const float* wx1, const float* wy1, const float* wz1,
                                              const float* __restrict__ F2, int x2, int y2, int z2,
                                              const float* wx2, const float* wy2, const float* wz2)
{
    float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int c = 0; c < NW; ++c) {
#pragma unroll
        for (int b = 0; b < NW; ++b) {
            const float* r1 = F1 + ((z1 + c) * TY + (y1 + b)) * PX + x1;
            const float* r2 = F2 + ((z2 + c) * TY + (y2 + b)) * PX + x2;
            float2 r = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int a = 0; a < NW; ++a)
                r = __ffma2_rn(make_float2(r1[a], r2[a]), make_float2(wx1[a], wx2[a]), r);
            acc = __ffma2_rn(r, __fmul2_rn(make_float2(wy1[b], wy2[b]), make_float2(wz1[c], wz2[c])), acc);
        }
    }
    return acc;
}

// Esirkepov transverse factor S0e S0f + (DSe S0f + S0e DSf)/2 + DSe DSf / 3.
__device__ __forceinline__ float esk_T(float s0e, float dse, float s0f, float dsf)
{
    return fmaf(s0e, s0f, fmaf(0.5f, fmaf(dse, s0f, s0e * dsf), (1.0f / 3.0f) * dse * dsf));
}

// ------------------------------------------------------------ fixed-point J tile
//
// The shared J tile accumulates each chunk of particles in int32: shared-
// memory int32 atomics are native, where FP32 shared atomics are a
// compare-and-swap loop.  A chunk's contributions are scaled by a power of
// two chosen from the chunk itself: with B = max over its particles and
// axes of Tmax |jcoef_d w D_d| (|P| <= |D| and |T| <= Tmax = (max S)^2 bound
// every term of the current by it) and n <= 256 particles, each scaled term is below 2^21 and a
// node's sum below 2^30, so nothing overflows and a term keeps 2^-22 B
// resolution.
// After the chunk the integer tile is folded into an FP32 tile.  Scaled terms
// convert to integers with the 1.5 * 2^23 magic-number add.
__device__ __forceinline__ int magic_int(float x)
{
    return __float_as_int(x + 12582912.0f) - 0x4B400000;
}

// scale = 2^(min(21, 30 - ceil(log2 n)) - e) with bound <= 2^e: a scaled
// term is below 2^21 (magic-number range) and n of them below 2^30
__device__ __forceinline__ float chunk_scale(int n, float bound, float* inv)
{
    const int lg = n > 1 ? 32 - __clz(n - 1) : 0;
    const int hb = min(21, 30 - lg);
    int e = 0;
    if (bound > 0.0f)
        frexpf(bound, &e);
    *inv = ldexpf(1.0f, e - hb);
    return ldexpf(1.0f, hb - e);
}

// Esirkepov factor of two lines at once (packed FP32; per lane the same
// operations as esk_T).
__device__ __forceinline__ float2 esk_T2(float2 s0e, float2 dse, float2 s0f, float2 dsf)
{
    const float2 half = make_float2(0.5f, 0.5f), third = make_float2(1.0f / 3.0f, 1.0f / 3.0f);
    return __ffma2_rn(s0e, s0f,
                      __ffma2_rn(half, __ffma2_rn(dse, s0f, __fmul2_rn(s0e, dsf)),
                                 __fmul2_rn(__fmul2_rn(third, dse), dsf)));
}

__device__ __forceinline__ float2 dup2(float v) { return make_float2(v, v); }

// One window line pair: the M - 1 terms P[i] T of two parallel lines (tile
// words a0 + i st and a1 + i st), converted to fixed point two at a time.
template <int M>
__device__ __forceinline__ void add_line_pair(int* a0, int* a1, int st, const float* P, float2 T)
{
    const float2 magic = dup2(12582912.0f);
#pragma unroll
    for (int i = 0; i < M - 1; ++i) {
        const float2 v = __ffma2_rn(dup2(P[i]), T, magic);
        atomicAdd(a0 + i * st, __float_as_int(v.x) - 0x4B400000);
        atomicAdd(a1 + i * st, __float_as_int(v.y) - 0x4B400000);
    }
}

// Deposit the three current components on a window of M nodes per axis
// (M-1 half nodes along the current's own axis); node 0 of axis d sits at
// tile index b[d].  cx..cz carry jcoef_d w times the chunk scale.  With
// PAIR (PCS: 144 atomics per move) the transverse factors and the
// fixed-point conversions go two lines at a time through the packed FP32
// pipe; for CIC and TSC the pairs' extra registers cost more than they save.
template <int M, int PX, int TY, int NJ, bool PAIR>
__device__ __forceinline__ void deposit_window(int* sJi, const int b[3], const float* S0x,
                                               const float* S0y, const float* S0z, const float* DSx,
                                               const float* DSy, const float* DSz, float cx, float cy,
                                               float cz)
{
    constexpr int PY = PX * TY;
    {
        float P[M - 1];
        P[0] = DSx[0];
#pragma unroll
        for (int i = 1; i < M - 1; ++i)
            P[i] = P[i - 1] + DSx[i];
#pragma unroll
        for (int k = 0; k < M; ++k)
#pragma unroll
            for (int j = 0; j < M; j += 2) {
                int* row = sJi + (b[2] + k) * PY + (b[1] + j) * PX + b[0];
                if (PAIR && j + 1 < M) {
                    const float2 T = __fmul2_rn(dup2(cx), esk_T2(make_float2(S0y[j], S0y[j + 1]),
                                                                make_float2(DSy[j], DSy[j + 1]),
                                                                dup2(S0z[k]), dup2(DSz[k])));
                    add_line_pair<M>(row, row + PX, 1, P, T);
                } else {
#pragma unroll
                    for (int jj = j; jj < (PAIR ? j + 1 : min(j + 2, M)); ++jj) {
                        const float T = cx * esk_T(S0y[jj], DSy[jj], S0z[k], DSz[k]);
                        int* r = row + (jj - j) * PX;
#pragma unroll
                        for (int i = 0; i < M - 1; ++i)
                            atomicAdd(r + i, magic_int(P[i] * T));
                    }
                }
            }
    }
    {
        float P[M - 1];
        P[0] = DSy[0];
#pragma unroll
        for (int i = 1; i < M - 1; ++i)
            P[i] = P[i - 1] + DSy[i];
#pragma unroll
        for (int k = 0; k < M; ++k)
#pragma unroll
            for (int i = 0; i < M; i += 2) {
                int* col = sJi + NJ + (b[2] + k) * PY + b[1] * PX + (b[0] + i);
                if (PAIR && i + 1 < M) {
                    const float2 T = __fmul2_rn(dup2(cy), esk_T2(dup2(S0z[k]), dup2(DSz[k]),
                                                                make_float2(S0x[i], S0x[i + 1]),
                                                                make_float2(DSx[i], DSx[i + 1])));
                    add_line_pair<M>(col, col + 1, PX, P, T);
                } else {
#pragma unroll
                    for (int ii = i; ii < (PAIR ? i + 1 : min(i + 2, M)); ++ii) {
                        const float T = cy * esk_T(S0z[k], DSz[k], S0x[ii], DSx[ii]);
                        int* c = col + (ii - i);
#pragma unroll
                        for (int j = 0; j < M - 1; ++j)
                            atomicAdd(c + j * PX, magic_int(P[j] * T));
                    }
                }
            }
    }
    {
        float P[M - 1];
        P[0] = DSz[0];
#pragma unroll
        for (int i = 1; i < M - 1; ++i)
            P[i] = P[i - 1] + DSz[i];
#pragma unroll
        for (int j = 0; j < M; ++j)
#pragma unroll
            for (int i = 0; i < M; i += 2) {
                int* col = sJi + 2 * NJ + b[2] * PY + (b[1] + j) * PX + (b[0] + i);
                if (PAIR && i + 1 < M) {
                    const float2 T = __fmul2_rn(dup2(cz), esk_T2(make_float2(S0x[i], S0x[i + 1]),
                                                                make_float2(DSx[i], DSx[i + 1]),
                                                                dup2(S0y[j]), dup2(DSy[j])));
                    add_line_pair<M>(col, col + 1, PY, P, T);
                } else {
#pragma unroll
                    for (int ii = i; ii < (PAIR ? i + 1 : min(i + 2, M)); ++ii) {
                        const float T = cz * esk_T(S0x[ii], DSx[ii], S0y[j], DSy[j]);
                        int* c = col + (ii - i);
#pragma unroll
                        for (int k = 0; k < M - 1; ++k)
                            atomicAdd(c + k * PY, magic_int(P[k] * T));
                    }
                }
            }
    }
}

// ------------------------------------------------------------ async copies

// 16-byte global -> shared copy that bypasses the registers (completes at
// cp_async_wait_all of the issuing thread; a block barrier then publishes it).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// ------------------------------------------------------------ TMA and mbarriers
//
// The E/B tile of a supercell arrives by two tensor loads (one per field, all
// three components) that complete on a shared-memory mbarrier with a byte
// count.  One thread issues and waits; a block barrier then publishes the
// tile.  The wait is bounded: after kWaitCycles SM clocks it gives up, the
// kernel reports ST_TIMEOUT and the CTA stops taking work.  (The particle
// chunks, scattered over the frames of a list, keep 16-byte asynchronous
// copies from many threads: as bulk copies issued by one thread they measured
// 5 % (TSC) and 8 % (CIC) slower.)

// ------------------------------------------------------------ warp helpers

__device__ __forceinline__ int warp_aggregated_add(int* ctr)
{
    unsigned mask = __activemask();
    int lane = threadIdx.x & 31;
    int leader = __ffs(mask) - 1;
    int base = 0;
    if (lane == leader)
        base = atomicAdd(ctr, __popc(mask));
    base = __shfl_sync(mask, base, leader);
    return base + __popc(mask & ((1u << lane) - 1u));
}

// Exclusive prefix sum of cnt[0..K) into off[0..K) by one warp (lanes take
// contiguous ranges); the caller synchronises the block around it.
__device__ __forceinline__ void warp_exclusive_scan_counts(const int* cnt, int* off, int K)
{
    const int lane = threadIdx.x & 31;
    const int per = (K + 31) / 32;
    const int b0 = lane * per;
    int local = 0;
    for (int i = 0; i < per; ++i)
        local += (b0 + i < K) ? cnt[b0 + i] : 0;
    int x = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o)
            x += y;
    }
    int run = x - local;
    for (int i = 0; i < per; ++i)
        if (b0 + i < K) {
            off[b0 + i] = run;
            run += cnt[b0 + i];
        }
}

// ------------------------------------------------------------ shared state

// Particles of one chunk of a frame list, staged in shared memory in list
// order, plus their counting-sort permutation by nearest node.
template <int C, bool PCS>
struct Stage {
    int cell[C];
    float o[3][C];
    float u[3][C];
    float w[C];
    int pid[C];   // particle ids (only when tracked)
    int kr[C];    // key << 16 | rank within key
    int perm[C];  // sorted position -> chunk position
    int brk[PCS ? C : 1];  // PCS, by push position: bank << 16 | rank within the bank
};

// Deposit inputs of the chunk's moves, by sorted position s stored at slot
// rslot(s) = s + s / 32: the deposit reads them with a stride of
// kDepStride between lanes, and the skew puts the 32 lanes on 32 different
// banks.
__host__ __device__ constexpr int rslot(int s) { return s + (s >> 5); }

// PCS (144 atomics per common-window move): the chunk's moves are
// counting-sorted by the shared-memory bank of their window origin (every
// atomic of a common-window deposit lands there plus an offset shared by all
// lanes) and dealt over the deposit lanes: slot q takes bank-major position
// deal_pos(q), so the 32 lanes of a deposit group take every (C/32)-th
// position -- mostly 32 different banks.
template <int C>
__host__ __device__ constexpr int deal_slot(int p)
{
    return (p % (C / 32)) * 32 + p / (C / 32);
}
template <int C>
__host__ __device__ constexpr int deal_pos(int q)
{
    return (q & 31) * (C / 32) + (q >> 5);
}

template <int C>
struct Records {
    static constexpr int R = C + C / 32;
    int l[R];        // packed local cell lx | ly << 8 | lz << 16, bit 24: general window
    float o[3][R];   // old in-cell offsets
    float D[3][R];   // displacement in cells
    float w[R];      // weight
    int gen[C];      // sorted positions of the moves that need the general window
};

template <class T, int SHAPE>
struct Keys {
    static constexpr int K = SHAPE == 2 ? (T::LX + 1) * (T::LY + 1) * (T::LZ + 1) : T::S;
};

template <class T>
constexpr int max_keys()
{
    return (T::LX + 1) * (T::LY + 1) * (T::LZ + 1);
}

// General-window moves set aside for one lane-parallel deposit after the
// last chunk of a frame list (the few of each chunk would otherwise keep one
// warp busy while the others wait at the chunk's last barrier).
struct GenDefer {
    int l[kGenDefer];        // packed local cell, as in Records
    float o[3][kGenDefer];   // old in-cell offsets
    float D[3][kGenDefer];   // displacement in cells
    float w[kGenDefer];      // weight
};

// Particles leaving the supercell, bound for the move buffer.
struct LeaverBuf {
    int dest[kLeaverBuf];  // destination list
    int cell[kLeaverBuf];  // cell inside the destination supercell
    float o[3][kLeaverBuf];
    float u[3][kLeaverBuf];
    float w[kLeaverBuf];
    int pid[kLeaverBuf];
};

template <class T, int NT>
struct SharedState {
    static constexpr int C = 2 * NT < 256 ? 2 * NT : 256;  // chunk: at most 256 particles
    static constexpr int NQ = C / NT;                       // particles per thread and chunk
    Stage<C, T::G == 2> st;
    Records<C> rec;
    GenDefer gd;
    LeaverBuf lv;
    int hist[max_keys<T>()];
    int off[max_keys<T>()];
    unsigned long long mb_tile;    // completion of the E/B tile's tensor loads
    unsigned alive[NQ * NT / 32];  // per warp and pass: ballot of the pushed particles that stay
    int item, any, nlv, lv_base;
    int tile_phase;                // parity of the tile barrier's next phase
    int abort;                     // the tile wait gave up
    int ngen[2];             // general-window moves of the chunk
    unsigned bound_bits[2];  // float bits of the chunk's largest |jcoef w D|
    unsigned gd_bound_bits;  // float bits of the largest |jcoef w D| of the set-aside moves
    int bh[T::G == 2 ? 32 : 1];  // PCS: moves of the chunk per bank of their window origin
};

// Bank of the common-window origin of a PCS particle in local cell `cell`
// (up to an offset shared by all particles).
template <class T>
__device__ __forceinline__ int dep_bank(int cell)
{
    const int lx = cell % T::LX, ly = (cell / T::LX) % T::LY, lz = cell / (T::LX * T::LY);
    return ((lz * T::TY + ly) * T::PX + lx) & 31;
}

// Exclusive prefix of the per-bank counts, bank `lane` in lane `lane`.
__device__ __forceinline__ int bank_offsets(const int* bh, int lane)
{
    const int c = bh[lane];
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o)
            incl += t;
    }
    return incl - c;
}

// Record slot of the move at push position sidx (all 32 lanes call it).
template <int C>
__device__ __forceinline__ int dealt_slot(const int* brk, int sidx, int cn, int boff)
{
    const int br = sidx < cn ? brk[sidx] : 0;
    return deal_slot<C>(__shfl_sync(0xffffffffu, boff, br >> 16) + (br & 0xffff));
}

// Stored-order passes: start copying the particles of list slots
// [base, base + cn) into the chunk stage (cell, offsets, momenta, weight;
// 16-byte pieces of whole frames, which are allocated even past the list's
// count).  The caller waits with cp_async_wait_all and a block barrier.
template <class T, int NT>
__device__ __forceinline__ void stage_chunk_async(const StepDev& d, SharedState<T, NT>& sh, int L, int base,
                                                  int cn)
{
    constexpr int S = T::S;
    const int* ft = d.ftab + d.foff[L];
    const int nq = (cn + 3) >> 2;
    for (int k = threadIdx.x; k < nq; k += NT) {
        const int slot = base + 4 * k;
        const int64_t idx = (int64_t)ft[slot >> d.log2S] * S + (slot & (S - 1));
        cp_async16(sh.st.cell + 4 * k, d.cell + idx);
        cp_async16(sh.st.o[0] + 4 * k, d.ox + idx);
        cp_async16(sh.st.o[1] + 4 * k, d.oy + idx);
        cp_async16(sh.st.o[2] + 4 * k, d.oz + idx);
        cp_async16(sh.st.u[0] + 4 * k, d.ux + idx);
        cp_async16(sh.st.u[1] + 4 * k, d.uy + idx);
        cp_async16(sh.st.u[2] + 4 * k, d.uz + idx);
        cp_async16(sh.st.w + 4 * k, d.w + idx);
    }
}

// ------------------------------------------------------------ deposit of one record

// Common window: nodes a-1, a, a+1 (TSC, a = round(o)), 0, 1 (CIC) or -1 .. 2
// (PCS) relative to the cell on every axis; S0 is the particle's shape there
// and DS has closed forms in D.  The record's l holds cell + GO per axis.
template <class T, int SHAPE, int C>
__device__ __forceinline__ void deposit_common(int* sJi, const Records<C>& r, int s, const float jc[3],
                                               float scale)
{
    const int e = rslot(s);
    constexpr int NW = SHAPE == 2 ? 3 : (SHAPE == 3 ? 4 : 2);
    const int l = r.l[e];
    const int lc[3] = {l & 0xff, (l >> 8) & 0xff, (l >> 16) & 0xff};
    float S0[3][NW], DS[3][NW];
    int b[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float o = r.o[a][e], D = r.D[a][e];
        if (SHAPE == 2) {
            const bool up = o >= 0.5f;
            const float di = up ? o - 1.0f : o;
            b[a] = lc[a] + (up ? 1 : 0);
            const float lo = 0.5f - di, hi = 0.5f + di;
            S0[a][0] = 0.5f * lo * lo;
            S0[a][1] = 0.75f - di * di;
            S0[a][2] = 0.5f * hi * hi;
            // DS = -D/2 (1 - d0 - d1), -D (d0 + d1), D/2 (1 + d0 + d1), d1 = d0 + D
            const float sum = 2.0f * di + D;
            DS[a][0] = -0.5f * D * (1.0f - sum);
            DS[a][1] = -D * sum;
            DS[a][2] = 0.5f * D * (1.0f + sum);
        } else if (SHAPE == 3) {
            // nodes cell-1 .. cell+2, each on one spline piece for the whole move:
            // outer (a = 1 - o), centre (d = o), centre (d = o - 1), outer (a = o)
            b[a] = lc[a];
            const float o1 = o + D;
            const float a0 = 1.0f - o, a1 = a0 - D;
            const float d0 = o - 1.0f, d1 = o1 - 1.0f;
            S0[a][0] = a0 * a0 * a0 * (1.0f / 6.0f);
            S0[a][1] = (4.0f - 6.0f * o * o + 3.0f * o * o * o) * (1.0f / 6.0f);
            S0[a][2] = (4.0f - 6.0f * d0 * d0 - 3.0f * d0 * d0 * d0) * (1.0f / 6.0f);
            S0[a][3] = o * o * o * (1.0f / 6.0f);
            DS[a][0] = -D * (a0 * a0 + a0 * a1 + a1 * a1) * (1.0f / 6.0f);
            DS[a][1] = D * (-(o + o1) + 0.5f * (o * o + o * o1 + o1 * o1));
            DS[a][2] = D * (-(d0 + d1) - 0.5f * (d0 * d0 + d0 * d1 + d1 * d1));
            DS[a][3] = D * (o * o + o * o1 + o1 * o1) * (1.0f / 6.0f);
        } else {
            b[a] = lc[a] + 1;
            S0[a][0] = 1.0f - o;
            S0[a][1] = o;
            DS[a][0] = -D;
            DS[a][1] = D;
        }
    }
    const float ws = r.w[e] * scale;
    deposit_window<NW, T::PX, T::TY, T::N, SHAPE == 3>(sJi, b, S0[0], S0[1], S0[2], DS[0], DS[1], DS[2], jc[0] * ws,
                                           jc[1] * ws, jc[2] * ws);
}

// Window of the general deposit: M nodes per axis; on axis a its first node
// sits at tile index lc + first_off(o, D) and node k of the window is at
// distance d0 = o - node_off(o, D, k) from the particle.
template <int SHAPE>
struct GenWin {
    static constexpr int M = SHAPE == 3 ? 5 : 4;
    // PCS: nodes cell-2+up .. cell+2+up, up = the move ends in the next cell;
    // CIC / TSC: nodes cell-1 .. cell+2
    __device__ __forceinline__ static int first(float o, float D) { return SHAPE == 3 ? (o + D >= 1.0f) - 1 : 0; }
    __device__ __forceinline__ static float d0(float o, int first, int k) { return o - (float)(k - 1 + first); }
    __device__ __forceinline__ static float S(float d) { return SHAPE == 3 ? pcs_S(d) : (SHAPE == 2 ? tsc_S(d) : cic_S(d)); }
    __device__ __forceinline__ static float dS(float d, float D)
    {
        return SHAPE == 3 ? pcs_dS(d, D) : (SHAPE == 2 ? tsc_dS(d, D) : cic_dS(d, D));
    }
};

// General window (GenWin) on every axis, for the move of packed local cell
// l, old offsets o and displacement D (in cells) of a particle of weight w.
template <class T, int SHAPE>
__device__ __forceinline__ void deposit_general_move(int* sJi, int l, const float ov[3], const float Dv[3],
                                                     float w, const float jc[3], float scale)
{
    using W = GenWin<SHAPE>;
    constexpr int M = W::M;
    const int lc[3] = {l & 0xff, (l >> 8) & 0xff, (l >> 16) & 0xff};  // node cell-1 sits at tile index lc
    float S0[3][M], DS[3][M];
    int b[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float o = ov[a], D = Dv[a];
        const int f = W::first(o, D);
        b[a] = lc[a] + f;
#pragma unroll
        for (int k = 0; k < M; ++k) {
            const float d0 = W::d0(o, f, k);
            S0[a][k] = W::S(d0);
            DS[a][k] = W::dS(d0, D);
        }
    }
    const float ws = w * scale;
    deposit_window<M, T::PX, T::TY, T::N, SHAPE == 3>(sJi, b, S0[0], S0[1], S0[2], DS[0], DS[1], DS[2], jc[0] * ws,
                                          jc[1] * ws, jc[2] * ws);
}

// The general-window move at sorted position s of the chunk's records.
template <class T, int SHAPE, int C>
__device__ __forceinline__ void deposit_general(int* sJi, const Records<C>& r, int s, const float jc[3],
                                                float scale)
{
    const int e = rslot(s);
    const float o[3] = {r.o[0][e], r.o[1][e], r.o[2][e]};
    const float D[3] = {r.D[0][e], r.D[1][e], r.D[2][e]};
    deposit_general_move<T, SHAPE>(sJi, r.l[e], o, D, r.w[e], jc, scale);
}

// Bound on the current terms of one move (see push_one).
template <int SHAPE>
__device__ __forceinline__ float move_bound(const float jc[3], float w, float Dx, float Dy, float Dz)
{
    const float tmax = SHAPE == 2 ? 0.5625f * 1.001f : (SHAPE == 3 ? (4.0f / 9.0f) * 1.001f : 1.0f);
    return tmax * fabsf(w) * fmaxf(fmaxf(fabsf(jc[0] * Dx), fabsf(jc[1] * Dy)), fabsf(jc[2] * Dz));
}

// General window of one move, deposited by a whole warp (all 32 lanes
// converged): lane 8a + k (k < M) evaluates S0 and DS at node k of axis a's
// window and the prefix P of DS along that axis; then the lanes take the
// window's 3 M^2 lines (a component c and its transverse nodes p, q: M - 1
// half nodes along c) in turns, reading the factors they need from the
// lanes that hold them.
template <class T, int SHAPE, int C>
__device__ __forceinline__ void deposit_general_warp(int* sJi, const Records<C>& r, int s,
                                                     const float jc[3], float scale)
{
    using W = GenWin<SHAPE>;
    constexpr int M = W::M;
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int PX = T::PX, PY = T::PX * T::TY, NJ = T::N;
    const int lane = threadIdx.x & 31;
    const int e = rslot(s);
    const int l = r.l[e];
    int f[3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
        f[a] = W::first(r.o[a][e], r.D[a][e]);  // same address in every lane: broadcasts
    float s0v = 0.0f, dsv = 0.0f;
    if ((lane & 7) < M && lane < 24) {
        const int a = lane >> 3, k = lane & 7;
        const float o = r.o[a][e], D = r.D[a][e];
        const float d0 = W::d0(o, a == 0 ? f[0] : (a == 1 ? f[1] : f[2]), k);
        s0v = W::S(d0);
        dsv = W::dS(d0, D);
    }
    float pv = dsv;  // inclusive prefix over k within each group of 8 lanes
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
        const float t = __shfl_up_sync(FULL, pv, o, 8);
        if ((lane & 7) >= o)
            pv += t;
    }
    const float ws = r.w[e] * scale;
    const int b0 = (l & 0xff) + f[0], b1 = ((l >> 8) & 0xff) + f[1], b2 = ((l >> 16) & 0xff) + f[2];
    const int base = b2 * PY + b1 * PX + b0;
    constexpr int LINES = 3 * M * M;
#pragma unroll
    for (int round = 0; round < (LINES + 31) / 32; ++round) {
        const int L = lane + 32 * round;  // c = L / M^2, p = L % M, q = (L / M) % M
        const int c = L / (M * M);
        const int ea = c == 2 ? 0 : c + 1, fa = c == 0 ? 2 : c - 1;  // transverse axes
        const int p = L % M, q = (L / M) % M;
        const int srcE = 8 * ea + p, srcF = 8 * fa + q;
        const float s0e = __shfl_sync(FULL, s0v, srcE & 31), dse = __shfl_sync(FULL, dsv, srcE & 31);
        const float s0f = __shfl_sync(FULL, s0v, srcF & 31), dsf = __shfl_sync(FULL, dsv, srcF & 31);
        float P[M - 1];
#pragma unroll
        for (int i = 0; i < M - 1; ++i)
            P[i] = __shfl_sync(FULL, pv, (8 * c + i) & 31);
        if (L < LINES) {
            const float cf = (c == 0 ? jc[0] : (c == 1 ? jc[1] : jc[2])) * ws;
            const float Tv = cf * esk_T(s0e, dse, s0f, dsf);
            const int st_c = c == 0 ? 1 : (c == 1 ? PX : PY);
            const int st_e = ea == 0 ? 1 : (ea == 1 ? PX : PY);
            const int st_f = fa == 0 ? 1 : (fa == 1 ? PX : PY);
            int* at = sJi + c * NJ + base + p * st_e + q * st_f;
#pragma unroll
            for (int i = 0; i < M - 1; ++i)
                atomicAdd(at + i * st_c, magic_int(P[i] * Tv));
        }
    }
}

// ------------------------------------------------------------ one particle

// One particle in registers.
struct Part {
    int cell;
    float o[3], u[3], w;
};

// Writes a pushed particle to pool slot idx (only the cell of a leaver);
// the weight only when the particle changed slot.
__device__ __forceinline__ void store_part(const StepDev& d, int64_t idx, const Part& q, bool with_w)
{
    d.cell[idx] = q.cell;
    if (q.cell >= 0) {
        d.ox[idx] = q.o[0];
        d.oy[idx] = q.o[1];
        d.oz[idx] = q.o[2];
        d.ux[idx] = q.u[0];
        d.uy[idx] = q.u[1];
        d.uz[idx] = q.u[2];
        if (with_w)
            d.w[idx] = q.w;
    }
}

// Pushes one particle (gather, Boris, move) and writes its deposit record
// at slot `slot` of the chunk; returns its bound |jcoef_d w D_d| on the
// current terms.  A particle that stays in the supercell gets its new cell,
// offsets and momentum in q; a leaver goes to the CTA's leaver buffer (or,
// when that is full, straight to the move buffer), to a neighbouring slab's
// migrant message, or out of an open-y box; its id is `pid` when ids are
// tracked, and q.cell becomes -1.
template <class T, int SHAPE, int NT>
__device__ __forceinline__ float push_one(const StepDev& d, const SpeciesDev& sp, int s, const BoxDev& bx,
                                         int scx, int scy, int scz, const float* sF,
                                         SharedState<T, NT>& sh, Part& q, int pid,
                                         int slot, int cb, unsigned& my_status)
{
    constexpr int LX = T::LX, LY = T::LY, LZ = T::LZ, N = T::N, PX = T::PX, TY = T::TY;
    constexpr int NW = SHAPE == 2 ? 3 : (SHAPE == 3 ? 4 : 2);
    constexpr int GO = T::GO;
    auto& rec = sh.rec;
    const int cell = q.cell;
    const float ox = q.o[0], oy = q.o[1], oz = q.o[2];
    float ux = q.u[0], uy = q.u[1], uz = q.u[2];
    const float w = q.w;
    const int lx = cell % LX;
    const int ly = (cell / LX) % LY;
    const int lz = cell / (LX * LY);

    // gather (Sec. 4: product of 1D weights at each Yee position)
    const bool ec = sp.ec != 0;
    AxisW<SHAPE> ax(lx + GO, ox, ec), ay(ly + GO, oy, ec), az(lz + GO, oz, ec);
    // TSC and PCS: two components per packed FP32 instruction; CIC (8 terms
    // a component) keeps the scalar form, which measured faster there
    float Ex, Ey, Ez, Bx, By, Bz;
    if constexpr (SHAPE != 1) {
        const float2 Exy = gather_pair<NW, PX, TY>(sF + 0 * N, ax.bh, ay.bi, az.bi, ax.wh, ay.wi, az.wi,
                                                   sF + 1 * N, ax.bi, ay.bh, az.bi, ax.wi, ay.wh, az.wi);
        const float2 EzBx = gather_pair<NW, PX, TY>(sF + 2 * N, ax.bi, ay.bi, az.bh, ax.wi, ay.wi, az.wh,
                                                    sF + T::BOFF, ax.bi, ay.bh, az.bh, ax.wi, ay.wh, az.wh);
        const float2 Byz = gather_pair<NW, PX, TY>(sF + T::BOFF + N, ax.bh, ay.bi, az.bh, ax.wh, ay.wi, az.wh,
                                                   sF + T::BOFF + 2 * N, ax.bh, ay.bh, az.bi, ax.wh, ay.wh, az.wi);
        Ex = Exy.x, Ey = Exy.y, Ez = EzBx.x, Bx = EzBx.y, By = Byz.x, Bz = Byz.y;
    } else {
        Ex = gather_comp<NW, PX, TY>(sF + 0 * N, ax.bh, ay.bi, az.bi, ax.wh, ay.wi, az.wi);
        Ey = gather_comp<NW, PX, TY>(sF + 1 * N, ax.bi, ay.bh, az.bi, ax.wi, ay.wh, az.wi);
        Ez = gather_comp<NW, PX, TY>(sF + 2 * N, ax.bi, ay.bi, az.bh, ax.wi, ay.wi, az.wh);
        Bx = gather_comp<NW, PX, TY>(sF + T::BOFF, ax.bi, ay.bh, az.bh, ax.wi, ay.wh, az.wh);
        By = gather_comp<NW, PX, TY>(sF + T::BOFF + N, ax.bh, ay.bi, az.bh, ax.wh, ay.wi, az.wh);
        Bz = gather_comp<NW, PX, TY>(sF + T::BOFF + 2 * N, ax.bh, ay.bh, az.bi, ax.wh, ay.wh, az.wi);
    }

    // relativistic Boris push (Boris 1970): half kick, rotation, half kick
    const float eps = sp.eps;
    const float umx = fmaf(eps, Ex, ux), umy = fmaf(eps, Ey, uy), umz = fmaf(eps, Ez, uz);
    const float ginv = rsqrtf(1.0f + umx * umx + umy * umy + umz * umz);
    const float tx = eps * Bx * ginv, ty = eps * By * ginv, tz = eps * Bz * ginv;
    const float f = 2.0f / (1.0f + tx * tx + ty * ty + tz * tz);
    const float sx = f * tx, sy = f * ty, sz = f * tz;
    const float upx = umx + (umy * tz - umz * ty);
    const float upy = umy + (umz * tx - umx * tz);
    const float upz = umz + (umx * ty - umy * tx);
    ux = umx + (upy * sz - upz * sy) + eps * Ex;
    uy = umy + (upz * sx - upx * sz) + eps * Ey;
    uz = umz + (upx * sy - upy * sx) + eps * Ez;
    const float gi = rsqrtf(1.0f + ux * ux + uy * uy + uz * uz);
    float Dx = d.move[0] * ux * gi, Dy = d.move[1] * uy * gi, Dz = d.move[2] * uz * gi;
    if (!(fabsf(Dx) < 0.5f && fabsf(Dy) < 0.5f && fabsf(Dz) < 0.5f)) {
        my_status |= ST_PARTICLE;  // non-finite or superluminal: freeze it
        Dx = Dy = Dz = 0.0f;
        ux = uy = uz = 0.0f;
    }
    const float x1 = ox + Dx, y1 = oy + Dy, z1 = oz + Dz;

    // deposit record (the current goes in afterwards, in another lane order)
    bool common;
    if (SHAPE == 2)
        common = ((ox >= 0.5f) == (x1 >= 0.5f)) && ((oy >= 0.5f) == (y1 >= 0.5f)) &&
                 ((oz >= 0.5f) == (z1 >= 0.5f));
    else
        common = x1 >= 0.0f && x1 < 1.0f && y1 >= 0.0f && y1 < 1.0f && z1 >= 0.0f && z1 < 1.0f;
    const int rs = rslot(slot);
    rec.l[rs] = (lx + GO) | ((ly + GO) << 8) | ((lz + GO) << 16) | (common ? 0 : (1 << 24));
    rec.o[0][rs] = ox;
    rec.o[1][rs] = oy;
    rec.o[2][rs] = oz;
    rec.D[0][rs] = Dx;
    rec.D[1][rs] = Dy;
    rec.D[2][rs] = Dz;
    rec.w[rs] = w;
    if (!common)
        rec.gen[atomicAdd(&sh.ngen[cb], 1)] = slot;
    // bound on every current term of this particle: |jcoef_d w P| with |P| <= |D_d|
    // (P is a difference of cumulative shape sums, whose slope is at most 1),
    // times |T| <= (max S)^2: 9/16 for TSC (S <= 3/4), 4/9 for PCS (S <= 2/3), 1 for CIC
    const float bnd = move_bound<SHAPE>(sp.jcoef, w, Dx, Dy, Dz);

    // new cell and offsets
    const float fx_ = floorf(x1), fy_ = floorf(y1), fz_ = floorf(z1);
    const float kOneMinus = 0.99999994f;  // largest float below 1
    const float nox = fminf(x1 - fx_, kOneMinus);
    const float noy = fminf(y1 - fy_, kOneMinus);
    const float noz = fminf(z1 - fz_, kOneMinus);
    const int nlx = lx + (int)fx_, nly = ly + (int)fy_, nlz = lz + (int)fz_;
    const int dsx = nlx < 0 ? -1 : (nlx >= LX ? 1 : 0);
    const int dsy = nly < 0 ? -1 : (nly >= LY ? 1 : 0);
    const int dsz = nlz < 0 ? -1 : (nlz >= LZ ? 1 : 0);
    if ((dsx | dsy | dsz) == 0) {
        q.cell = nlx + LX * (nly + LY * nlz);
        q.o[0] = nox;
        q.o[1] = noy;
        q.o[2] = noz;
        q.u[0] = ux;
        q.u[1] = uy;
        q.u[2] = uz;
    } else {
        // leaves the supercell: into the move buffer, towards the neighbour
        // supercell (periodic within the box), or, through a y face of an
        // open-y box, out of the simulation
        int tsx = scx + dsx, tsy = scy + dsy, tsz = scz + dsz;
        if (bx.sub_z && (tsz < 0 || tsz >= bx.nscz)) {
            // through a z face of a subdomain slab: into that face's migrant
            // message for the neighbouring slab
            tsx += tsx < 0 ? bx.nscx : (tsx >= bx.nscx ? -bx.nscx : 0);
            tsy += tsy < 0 ? bx.nscy : (tsy >= bx.nscy ? -bx.nscy : 0);
            char* msg = d.mig + (tsz < 0 ? 0 : d.mig_bytes);
            const int m = atomicAdd(&reinterpret_cast<MigHeader*>(msg)->count, 1);
            if (m < d.mig_cap) {
                MigRec r;
                r.s = s;
                r.sx = tsx;
                r.sy = tsy;
                r.cell = (nlx - dsx * LX) + LX * ((nly - dsy * LY) + LY * (nlz - dsz * LZ));
                r.ox = nox;
                r.oy = noy;
                r.oz = noz;
                r.ux = ux;
                r.uy = uy;
                r.uz = uz;
                r.w = w;
                r.pid = pid;
                int4* dst = reinterpret_cast<int4*>(msg + sizeof(MigHeader) + (int64_t)m * sizeof(MigRec));
                const int4* src = reinterpret_cast<const int4*>(&r);
                dst[0] = src[0];
                dst[1] = src[1];
                dst[2] = src[2];
            } else {
                my_status |= ST_CAPACITY;
            }
        } else if (!(bx.oy.open_y && (tsy < 0 || tsy >= bx.nscy))) {
            tsx += tsx < 0 ? bx.nscx : (tsx >= bx.nscx ? -bx.nscx : 0);
            tsy += tsy < 0 ? bx.nscy : (tsy >= bx.nscy ? -bx.nscy : 0);
            tsz += tsz < 0 ? bx.nscz : (tsz >= bx.nscz ? -bx.nscz : 0);
            const int dest_sc = bx.sc_base + (tsz * bx.nscy + tsy) * bx.nscx + tsx;
            const int dest_cell = (nlx - dsx * LX) + LX * ((nly - dsy * LY) + LY * (nlz - dsz * LZ));
            const int destL = s * d.nsc + dest_sc;
            const int k = atomicAdd(&sh.nlv, 1);
            if (k < kLeaverBuf) {
                // handed to the move buffer at the CTA's next work item, so
                // that no warp waits here for a global atomic's reply
                sh.lv.dest[k] = destL;
                sh.lv.cell[k] = dest_cell;
                sh.lv.o[0][k] = nox;
                sh.lv.o[1][k] = noy;
                sh.lv.o[2][k] = noz;
                sh.lv.u[0][k] = ux;
                sh.lv.u[1][k] = uy;
                sh.lv.u[2][k] = uz;
                sh.lv.w[k] = w;
                sh.lv.pid[k] = pid;
            } else {
                const int m = warp_aggregated_add(d.mv_count);
                if (m < d.mv_cap) {
                    d.mv_rank[m] = atomicAdd(d.narrive + destL, 1);
                    d.mv_dest[m] = destL;
                    d.mv_cell[m] = dest_cell;
                    d.mv_ox[m] = nox;
                    d.mv_oy[m] = noy;
                    d.mv_oz[m] = noz;
                    d.mv_ux[m] = ux;
                    d.mv_uy[m] = uy;
                    d.mv_uz[m] = uz;
                    d.mv_w[m] = w;
                    if (d.pid)
                        d.mv_pid[m] = pid;
                } else {
                    my_status |= ST_CAPACITY;
                }
            }
        }
        q.cell = -1;
    }
    return bnd;
}

// The CTA's collected leavers into the move buffer: one reservation, then
// every leaver's rank among the arrivals of its destination list (all
// threads converged; sh.nlv stable since the last block barrier).
template <class T, int NT>
__device__ __forceinline__ void flush_leavers(const StepDev& d, SharedState<T, NT>& sh, unsigned& my_status)
{
    const int n = min(sh.nlv, kLeaverBuf);
    if (n == 0)
        return;
    if (threadIdx.x == 0)
        sh.lv_base = atomicAdd(d.mv_count, n);
    __syncthreads();
    const int base = sh.lv_base;
    for (int k = threadIdx.x; k < n; k += NT) {
        const int m = base + k;
        if (m >= d.mv_cap) {
            my_status |= ST_CAPACITY;
            continue;
        }
        const int L = sh.lv.dest[k];
        d.mv_rank[m] = atomicAdd(d.narrive + L, 1);
        d.mv_dest[m] = L;
        d.mv_cell[m] = sh.lv.cell[k];
        d.mv_ox[m] = sh.lv.o[0][k];
        d.mv_oy[m] = sh.lv.o[1][k];
        d.mv_oz[m] = sh.lv.o[2][k];
        d.mv_ux[m] = sh.lv.u[0][k];
        d.mv_uy[m] = sh.lv.u[1][k];
        d.mv_uz[m] = sh.lv.u[2][k];
        d.mv_w[m] = sh.lv.w[k];
        if (d.pid)
            d.mv_pid[m] = sh.lv.pid[k];
    }
}

// ------------------------------------------------------------ one frame list

// Add the chunk's integer tile (scaled back by inv) into the FP32 tile and
// clear it; each thread owns its entries (16-byte groups of four; N is a
// multiple of 4 and both tiles are 16-byte aligned), no atomics.
template <int N, int NT>
__device__ __forceinline__ void fold_tile(int* sJi, float* sJf, float inv)
{
    int4* qi = reinterpret_cast<int4*>(sJi);
    float4* qf = reinterpret_cast<float4*>(sJf);
    for (int v = threadIdx.x; v < 3 * N / 4; v += NT) {
        const int4 q = qi[v];
        if ((q.x | q.y | q.z | q.w) != 0) {
            float4 f = qf[v];
            f.x = fmaf((float)q.x, inv, f.x);
            f.y = fmaf((float)q.y, inv, f.y);
            f.z = fmaf((float)q.z, inv, f.z);
            f.w = fmaf((float)q.w, inv, f.w);
            qf[v] = f;
            qi[v] = make_int4(0, 0, 0, 0);
        }
    }
}

// Pushes the frame list of species s in supercell g chunk by chunk and
// deposits its current into the shared tile; returns the number of its
// particles that stay (the list's new count; they occupy its first slots).
template <class T, int SHAPE, int NT>
__device__ __forceinline__ int push_list(const StepDev& d, const SpeciesDev& sp, int s, int g,
                                          const BoxDev& bx, int scx, int scy, int scz,
                                          const float* sF, int* sJi, float* sJf,
                                          SharedState<T, NT>& sh, bool sort_pass, unsigned& my_status)
{
    constexpr int LX = T::LX, LY = T::LY, S = T::S, N = T::N;
    constexpr int C = SharedState<T, NT>::C;
    constexpr int K = Keys<T, SHAPE>::K;
    constexpr bool DEAL = SHAPE == 3;  // bank-dealt deposit slots (see deal_slot)
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int L = s * d.nsc + g;
    const int n = d.count[L];
    const int* ft = d.ftab + d.foff[L];
    auto gidx = [&](int slot) -> int64_t { return (int64_t)ft[slot >> d.log2S] * S + (slot & (S - 1)); };
    constexpr int NQ = SharedState<T, NT>::NQ, NWARP = NT / 32;
    float prev_inv = 0.0f;
    int ndef = 0;  // general-window moves set aside in sh.gd
    int surv = 0;  // particles of the list that stay, written back so far
    // chunk c uses the bound / general-list counters cb = c & 1; the other
    // pair is cleared after the chunk's first barrier (its last readers were
    // the previous chunk's deposits, its next writers come after the next
    // chunk's last barrier)
    int cb = 0;
    for (int base = 0; base < n; base += C, cb ^= 1) {
        const int cn = min(C, n - base);
        if (base > 0)
            fold_tile<N, NT>(sJi, sJf, prev_inv);  // previous chunk; the push below does not touch J
        int boff = 0;
        if (sort_pass) {
            // stage the chunk (coalesced), key = nearest node (TSC) / cell (CIC),
            // then a counting sort; the pushed particles go back to the list
            // in sorted order, so the list stays sorted by node between passes
            for (int k = tid; k < K; k += NT)
                sh.hist[k] = 0;
            __syncthreads();
            for (int j = tid; j < cn; j += NT) {
                const int64_t idx = gidx(base + j);
                const int cell = d.cell[idx];
                const float ox = d.ox[idx], oy = d.oy[idx], oz = d.oz[idx];
                sh.st.cell[j] = cell;
                sh.st.o[0][j] = ox;
                sh.st.o[1][j] = oy;
                sh.st.o[2][j] = oz;
                sh.st.u[0][j] = d.ux[idx];
                sh.st.u[1][j] = d.uy[idx];
                sh.st.u[2][j] = d.uz[idx];
                sh.st.w[j] = d.w[idx];
                if (d.pid)
                    sh.st.pid[j] = d.pid[idx];
                int key;
                if (SHAPE == 2) {
                    const int lx = cell % LX + (ox >= 0.5f), ly = (cell / LX) % LY + (oy >= 0.5f),
                              lz = cell / (LX * LY) + (oz >= 0.5f);
                    key = lx + (LX + 1) * (ly + (LY + 1) * lz);
                } else {
                    key = cell;
                }
                sh.st.kr[j] = (key << 16) | atomicAdd(&sh.hist[key], 1);
            }
            __syncthreads();
            if (wid == 0)
                warp_exclusive_scan_counts(sh.hist, sh.off, K);
            __syncthreads();
            for (int j = tid; j < cn; j += NT) {
                const int kr = sh.st.kr[j];
                const int ps = sh.off[kr >> 16] + (kr & 0xffff);
                sh.st.perm[ps] = j;
                if (DEAL) {
                    const int bk = dep_bank<T>(sh.st.cell[j]);
                    sh.st.brk[ps] = (bk << 16) | atomicAdd(&sh.bh[bk], 1);
                }
            }
            __syncthreads();
            boff = DEAL ? bank_offsets(sh.bh, lane) : 0;
        } else if (DEAL) {
            for (int j = tid; j < cn; j += NT) {
                const int bk = dep_bank<T>(sh.st.cell[j]);
                sh.st.brk[j] = (bk << 16) | atomicAdd(&sh.bh[bk], 1);
            }
            __syncthreads();
            boff = bank_offsets(sh.bh, lane);
        }
        // push: sort passes in sorted order (neighbouring lanes read
        // neighbouring field words), the passes between in stored order from
        // the stage an async copy filled while the previous chunk deposited.
        // Every read of the chunk's list slots happens before the barrier
        // below, every write after it.
        Part qs[NQ];
        int pids[NQ];
#pragma unroll
        for (int r = 0; r < NQ; ++r) {
            const int sidx = r * NT + tid;
            const int slot = DEAL ? dealt_slot<C>(sh.st.brk, sidx, cn, boff) : sidx;
            float bnd = 0.0f;
            qs[r].cell = -1;
            if (sidx < cn) {
                const int j = sort_pass ? sh.st.perm[sidx] : sidx;
                Part& q = qs[r];
                q.cell = sh.st.cell[j];
                q.o[0] = sh.st.o[0][j];
                q.o[1] = sh.st.o[1][j];
                q.o[2] = sh.st.o[2][j];
                q.u[0] = sh.st.u[0][j];
                q.u[1] = sh.st.u[1][j];
                q.u[2] = sh.st.u[2][j];
                q.w = sh.st.w[j];
                pids[r] = !d.pid ? 0 : (sort_pass ? sh.st.pid[j] : d.pid[gidx(base + sidx)]);
                bnd = push_one<T, SHAPE, NT>(d, sp, s, bx, scx, scy, scz, sF, sh, q, pids[r], slot, cb,
                                             my_status);
            }
            const unsigned stay = __ballot_sync(0xffffffffu, qs[r].cell >= 0);
            const unsigned m = __reduce_max_sync(0xffffffffu, __float_as_uint(bnd));
            if (lane == 0) {
                sh.alive[r * NWARP + wid] = stay;
                atomicMax(&sh.bound_bits[cb], m);
            }
        }
        __syncthreads();
        // the particles that stay go back to the list compacted, in chunk
        // order (the leavers' slots close up; sorted lists stay sorted)
        {
            int run = 0, pre[NQ];
#pragma unroll
            for (int r = 0; r < NQ; ++r)
                for (int w = 0; w < NWARP; ++w) {
                    if (w == wid)
                        pre[r] = run;
                    run += __popc(sh.alive[r * NWARP + w]);
                }
#pragma unroll
            for (int r = 0; r < NQ; ++r) {
                if (qs[r].cell < 0)
                    continue;
                const int src = base + r * NT + tid;
                const int dst = surv + pre[r] + __popc(sh.alive[r * NWARP + wid] & ((1u << lane) - 1u));
                const bool moved = sort_pass || dst != src;
                const int64_t idx = gidx(dst);
                store_part(d, idx, qs[r], moved);
                if (d.pid && moved)
                    d.pid[idx] = pids[r];
            }
            surv += run;
        }
        if (tid == 0) {
            sh.ngen[cb ^ 1] = 0;
            sh.bound_bits[cb ^ 1] = 0u;
        }
        if (DEAL && T::G == 2 && tid < 32)
            sh.bh[tid] = 0;  // every warp read it before the barrier above; next written after the chunk
        if (!sort_pass && base + C < n)  // the stage is free: the next chunk flies during the deposit
            stage_chunk_async<T, NT>(d, sh, L, base + C, min(C, n - base - C));
        // deposit: neighbouring lanes take chunk positions kDepStride apart
        // (sorted by node, so one warp's atomics land on different nodes and
        // mostly different banks); then the general-window moves
        float inv;
        const float scale = chunk_scale(cn, __uint_as_float(sh.bound_bits[cb]), &inv);
        for (int r = 0; r < C / NT; ++r) {
            const int q = r * NT + tid;
            const int e = DEAL ? q : kDepStride * (q % (C / kDepStride)) + q / (C / kDepStride);
            if ((DEAL ? deal_pos<C>(q) : e) < cn && !(sh.rec.l[rslot(e)] >> 24))
                deposit_common<T, SHAPE, C>(sJi, sh.rec, e, sp.jcoef, scale);
        }
        // general-window moves: set aside for the list's end while they fit
        // (ngen and ndef are the same in every thread); otherwise whole groups
        // of 32 lane-parallel, one group per warp, and the rest one move per
        // warp, all lanes on it
        const int ngen = sh.ngen[cb];
        if (ndef + ngen <= kGenDefer) {
            for (int q = tid; q < ngen; q += NT) {
                const int e = rslot(sh.rec.gen[q]);
                const int k = ndef + q;
                const float Dx = sh.rec.D[0][e], Dy = sh.rec.D[1][e], Dz = sh.rec.D[2][e], w = sh.rec.w[e];
                sh.gd.l[k] = sh.rec.l[e];
                sh.gd.o[0][k] = sh.rec.o[0][e];
                sh.gd.o[1][k] = sh.rec.o[1][e];
                sh.gd.o[2][k] = sh.rec.o[2][e];
                sh.gd.D[0][k] = Dx;
                sh.gd.D[1][k] = Dy;
                sh.gd.D[2][k] = Dz;
                sh.gd.w[k] = w;
                atomicMax(&sh.gd_bound_bits, __float_as_uint(move_bound<SHAPE>(sp.jcoef, w, Dx, Dy, Dz)));
            }
            ndef += ngen;
        } else {
            const int nfull = ngen & ~31;
            for (int q = tid; q < nfull; q += NT)
                deposit_general<T, SHAPE, C>(sJi, sh.rec, sh.rec.gen[q], sp.jcoef, scale);
            const int rem = ngen - nfull;
            for (int t = ((wid - (nfull >> 5)) % NWARP + NWARP) % NWARP; t < rem; t += NWARP)
                deposit_general_warp<T, SHAPE, C>(sJi, sh.rec, sh.rec.gen[nfull + t], sp.jcoef, scale);
        }
        prev_inv = inv;
        if (!sort_pass)
            cp_async_wait_all();
        __syncthreads();
    }
    if (n > 0)
        fold_tile<N, NT>(sJi, sJf, prev_inv);
    if (ndef > 0) {
        // the set-aside general-window moves, one per thread, with their own
        // fixed-point scale (at most kGenDefer terms per node)
        __syncthreads();
        float inv;
        const float scale = chunk_scale(ndef, __uint_as_float(sh.gd_bound_bits), &inv);
        for (int k = tid; k < ndef; k += NT) {
            const float o[3] = {sh.gd.o[0][k], sh.gd.o[1][k], sh.gd.o[2][k]};
            const float D[3] = {sh.gd.D[0][k], sh.gd.D[1][k], sh.gd.D[2][k]};
            deposit_general_move<T, SHAPE>(sJi, sh.gd.l[k], o, D, sh.gd.w[k], sp.jcoef, scale);
        }
        __syncthreads();
        fold_tile<N, NT>(sJi, sJf, inv);
    }
    // the caller synchronises before the flush
    return surv;
}

// ------------------------------------------------------------ the kernel

template <class T, int NT>
__global__ void __launch_bounds__(NT, (T::G == 1 ? 1024 : 512) / NT) k_push_deposit(const StepDev d)
{
    constexpr int TX = T::TX, TY = T::TY, TZ = T::TZ, PX = T::PX, N = T::N;
    constexpr int LX = T::LX, LY = T::LY, LZ = T::LZ;
    extern __shared__ __align__(128) float smem[];
    // layout (dyn_smem): [3N E floats, padded to BOFF][3N B floats][3N int current][3N float current]
    // [SharedState]
    float* sF = smem;  // [3][TZ][TY][PX] Ex Ey Ez at sF, Bx By Bz at sF + BOFF
    int* sJi = reinterpret_cast<int*>(smem + T::BOFF + 3 * N);  // [3][TZ][TY][PX] chunk accumulator
    float* sJf = smem + T::BOFF + 6 * N;                        // [3][TZ][TY][PX] supercell current
    SharedState<T, NT>& sh = *reinterpret_cast<SharedState<T, NT>*>(smem + T::TILES);

    const int tid = threadIdx.x;
    unsigned my_status = 0;
    // every sort_every-th step reorders the lists (the counter only changes
    // between launches, so all CTAs agree)
    const bool sort_pass = d.sort_every <= 1 || (*d.step_ctr % d.sort_every) == 0;

    // work items: tid 0 asks for the next one while the block works on the
    // current one, and publishes it at the end of the item
    if (tid == 0) {
        sh.item = atomicAdd(d.work_counter, 1);
        sh.nlv = 0;
        mbar_init(&sh.mb_tile, 1);
        fence_mbar_init();
        sh.tile_phase = 0;
        sh.abort = 0;
    }
    if (T::G == 2 && tid < 32)
        sh.bh[tid] = 0;  // each chunk clears it after use
    __syncthreads();
    for (;;) {
        const int item = sh.item;
        if (item >= d.nsc)
            break;
        int next_item = 0;
        if (tid == 0)
            next_item = atomicAdd(d.work_counter, 1);
        // the previous item's leavers into the move buffer (their global
        // atomics' replies come back while this item starts)
        flush_leavers<T, NT>(d, sh, my_status);
        const int g = d.items[item];
        const BoxDev bx = d.boxes[d.sc_box[g]];
        const int loc = g - bx.sc_base;
        const int scx = loc % bx.nscx;
        const int scy = (loc / bx.nscx) % bx.nscy;
        const int scz = loc / (bx.nscx * bx.nscy);

        if (tid == 0) {
            int ntot = 0;
            for (int s = 0; s < d.nspecies; ++s) {
                const int c = d.count[s * d.nsc + g];
                if (d.sp[s].mobile && c > 0)
                    ntot += c;
            }
            sh.any = ntot;
            sh.nlv = 0;  // every thread read it in flush_leavers (before its barrier, if it had one)
        }
        __syncthreads();
        if (sh.any == 0) {
            if (tid == 0)
                sh.item = next_item;
            __syncthreads();  // item / any are rewritten next round
            continue;
        }


        // ---- 1. the E/B tile by two tensor loads (TMA); on a stored-order
        // pass the first chunk of the first mobile list is copied meanwhile;
        // the next work item's tile is prefetched into L2; the J tiles are
        // zeroed
        int pre_s = -1;
        if (!sort_pass) {
            for (int s = 0; s < d.nspecies && pre_s < 0; ++s) {
                const int n = d.count[s * d.nsc + g];
                if (d.sp[s].mobile && n > 0) {
                    pre_s = s;
                    stage_chunk_async<T, NT>(d, sh, s * d.nsc + g, 0, min(SharedState<T, NT>::C, n));
                }
            }
        }
        if (tid == 0) {
            fence_proxy_async();
            mbar_expect_tx(&sh.mb_tile, 6u * 4u * (unsigned)N);
            const CUtensorMap* tm = d.tmaps + 2 * d.sc_box[g];
            tma_load_tile(sF, tm, scx * LX, scy * LY, scz * LZ, &sh.mb_tile);
            tma_load_tile(sF + T::BOFF, tm + 1, scx * LX, scy * LY, scz * LZ, &sh.mb_tile);
            if (next_item < d.nsc) {
                const int gn = d.items[next_item];
                const int bn = d.sc_box[gn];
                const BoxDev& bxn = d.boxes[bn];
                const int ln = gn - bxn.sc_base;
                const int xn = (ln % bxn.nscx) * LX, yn = ((ln / bxn.nscx) % bxn.nscy) * LY,
                          zn = (ln / (bxn.nscx * bxn.nscy)) * LZ;
                tma_prefetch_tile(d.tmaps + 2 * bn, xn, yn, zn);
                tma_prefetch_tile(d.tmaps + 2 * bn + 1, xn, yn, zn);
            }
        }
        for (int v = tid; v < 6 * N / 4; v += NT)  // int and float current tiles, contiguous; 0 bits = 0.0f
            reinterpret_cast<int4*>(sJi)[v] = make_int4(0, 0, 0, 0);
        if (tid == 0) {
            if (mbar_wait(&sh.mb_tile, (unsigned)sh.tile_phase)) {
                sh.tile_phase ^= 1;
            } else {
                sh.abort = 1;
                my_status |= ST_TIMEOUT;
            }
        }
        __syncthreads();
        if (sh.abort)
            break;

        // ---- 2. particles of every mobile species, 3. compaction
        for (int s = 0; s < d.nspecies; ++s) {
            const SpeciesDev sp = d.sp[s];
            const int L = s * d.nsc + g;
            const int n = d.count[L];
            if (!sp.mobile || n == 0)
                continue;
            if (tid == 0) {
                sh.ngen[0] = 0;
                sh.bound_bits[0] = 0u;
                sh.gd_bound_bits = 0u;
            }
            if (!sort_pass) {
                if (s != pre_s)
                    stage_chunk_async<T, NT>(d, sh, L, 0, min(SharedState<T, NT>::C, n));
                cp_async_wait_all();
            }
            __syncthreads();
            int stay;
            if (sp.shape == 2)
                stay = push_list<T, 2, NT>(d, sp, s, g, bx, scx, scy, scz, sF, sJi, sJf, sh, sort_pass, my_status);
            else if (T::G == 2 && sp.shape == 3)
                stay = push_list<T, T::G == 2 ? 3 : 1, NT>(d, sp, s, g, bx, scx, scy, scz, sF, sJi, sJf, sh,
                                                           sort_pass, my_status);
            else
                stay = push_list<T, 1, NT>(d, sp, s, g, bx, scx, scy, scz, sF, sJi, sJf, sh, sort_pass, my_status);
            if (tid == 0 && stay != n)
                d.count[L] = stay;  // the particles that stay fill the list's first slots
            __syncthreads();
        }

        // ---- 4. add the J tile to global J
        const int64_t pcell = padded_cells(bx);
        const int64_t start = ((int64_t)(scz * LZ) * bx.py + scy * LY) * bx.px + scx * LX;
        constexpr int ROW4 = TX / 4;
        constexpr int NJ4 = 3 * TZ * TY * ROW4;
        for (int v = tid; v < NJ4; v += NT) {
            const int r4 = v % ROW4;
            const int row = v / ROW4;
            const float4 val = *reinterpret_cast<const float4*>(sJf + row * PX + 4 * r4);
            if (val.x != 0.f || val.y != 0.f || val.z != 0.f || val.w != 0.f) {
                const int ty = row % TY;
                const int tz = (row / TY) % TZ;
                const int c = row / (TY * TZ);
                float* dst = bx.J + c * pcell + start + ((int64_t)tz * bx.py + ty) * bx.px + 4 * r4;
                atomicAdd(reinterpret_cast<float4*>(dst), val);
            }
        }
        if (tid == 0)
            sh.item = next_item;
        __syncthreads();
    }
    if (sh.abort) {
        // the tile wait gave up: give the loads in flight the same time once
        // more before the CTA's shared memory is released
        if (tid == 0)
            mbar_wait(&sh.mb_tile, (unsigned)sh.tile_phase);
    } else {
        flush_leavers<T, NT>(d, sh, my_status);
    }
    if (my_status)
        atomicOr(d.status, my_status);
}

// ------------------------------------------------------------ dispatch

template <class T, int NT>
static size_t dyn_smem()
{
    // field tile (6 N floats) + int and float current tiles (3 N each) + shared state
    return sizeof(float) * T::TILES + sizeof(SharedState<T, NT>);
}

// Sets the kernel's shared-memory limit and returns its resident CTAs per SM
// (call once, outside stream capture).
template <class T, int NT>
static cudaError_t configure_one(int* per_sm)
{
    auto kern = k_push_deposit<T, NT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)dyn_smem<T, NT>());
    if (e != cudaSuccess)
        return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kern, NT, dyn_smem<T, NT>());
}

template <class T, int NT>
static cudaError_t launch_one(const StepDev& d, int grid, cudaStream_t st)
{
    grid = min(max(grid, 1), max(1, d.nsc));
    k_push_deposit<T, NT><<<grid, NT, dyn_smem<T, NT>(), st>>>(d);
    return cudaGetLastError();
}

// (supercell edges, threads, guard): guard 1 for CIC/TSC contexts, 2 for
// contexts with a PCS species
#define PIC_PUSH_CASES(X)  \
    X(4, 4, 4, 64, 1)      \
    X(4, 4, 4, 128, 1)     \
    X(4, 4, 4, 256, 1)     \
    X(8, 4, 4, 128, 1)     \
    X(8, 4, 4, 256, 1)     \
    X(8, 8, 4, 128, 1)     \
    X(8, 8, 4, 256, 1)     \
    X(8, 8, 8, 256, 1)     \
    X(4, 4, 4, 128, 2)     \
    X(8, 4, 4, 256, 2)

size_t push_smem_bytes(int LX, int LY, int LZ, int threads, int guard)
{
#define X(a, b, c, t, g)                                                   \
    if (LX == a && LY == b && LZ == c && threads == t && guard == g)       \
        return dyn_smem<Tile<a, b, c, g>, t>();
    PIC_PUSH_CASES(X)
#undef X
    return 0;
}

void push_tile_box(int LX, int LY, int LZ, int guard, int* px, int* ty, int* tz)
{
#define X(a, b, c, t, g)                                                              \
    if (LX == a && LY == b && LZ == c && guard == g) {                                \
        *px = Tile<a, b, c, g>::PX;                                                   \
        *ty = Tile<a, b, c, g>::TY;                                                   \
        *tz = Tile<a, b, c, g>::TZ;                                                   \
        return;                                                                       \
    }
    PIC_PUSH_CASES(X)
#undef X
    *px = *ty = *tz = 0;
}

int push_supported(int LX, int LY, int LZ, int threads, int guard)
{
#define X(a, b, c, t, g) if (LX == a && LY == b && LZ == c && threads == t && guard == g) return 1;
    PIC_PUSH_CASES(X)
#undef X
    return 0;
}

cudaError_t configure_push(int LX, int LY, int LZ, int threads, int guard, int* per_sm)
{
#define X(a, b, c, t, g)                                                   \
    if (LX == a && LY == b && LZ == c && threads == t && guard == g)       \
        return configure_one<Tile<a, b, c, g>, t>(per_sm);
    PIC_PUSH_CASES(X)
#undef X
    return cudaErrorInvalidValue;
}

cudaError_t launch_push_deposit(const StepDev& d, int threads, int grid, cudaStream_t st)
{
#define X(a, b, c, t, g)                                                   \
    if (d.LX == a && d.LY == b && d.LZ == c && threads == t && d.guard == g) \
        return launch_one<Tile<a, b, c, g>, t>(d, grid, st);
    PIC_PUSH_CASES(X)
#undef X
    return cudaErrorInvalidValue;
}

}  // namespace pic
