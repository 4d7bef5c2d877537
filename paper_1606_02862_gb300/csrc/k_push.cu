// k_push.cu -- fused field gather, Boris push, move and Esirkepov current
// deposition for the mixed (int32 cell + FP32 offset) particle form.
//
// One CTA works on one supercell at a time (Sec. 2.1: a supercell maps to a
// block, its threads share the supercell's particles); CTAs are persistent
// and pull supercells from a work counter, so boxes of any size and
// occupancy share one launch.  Per supercell:
//   1. stage the E and B tile (supercell + 1 guard cell below, 3 (x) / 2
//      (y, z) above) from HBM into shared memory with 16-byte vector loads;
//   2. zero a shared J tile of the same extent;
//   3. every thread takes particles of the supercell's frame lists: gather
//      E, B from shared memory (CIC 2x2x2 / TSC 3x3x3 weights per component
//      at its Yee position, Sec. 4), relativistic Boris push, move, then
//      Esirkepov deposition (Sec. 4) into the shared J tile with shared
//      atomics; particles that leave the supercell go to the move buffer;
//   4. compact the frame list (fill the holes the leavers left);
//   5. add the J tile to the guard-padded global J with 16-byte vector
//      atomics (neighbouring supercells overlap in their guard cells).
//
// Esirkepov (2001): with 1D shape factors S0 (old) and S1 (new) on a common
// window and DS = S1 - S0, the x current on the half node i+1/2 is
//   Jx(i+1/2, j, k) = -(q w hx / (V dt)) * sum_{i' <= i} DSx(i')
//                     * [S0y S0z + DSy S0z / 2 + S0y DSz / 2 + DSy DSz / 3](j, k)
// i.e. an outer product of a prefix sum along x and a transverse factor.
//
// Particles are staged a chunk at a time in shared memory (coalesced loads
// and stores) and pushed in the order of a counting sort by nearest node, so
// the lanes of a warp read neighbouring field words and add to neighbouring
// current words.  The current tile accumulates in fixed point (see fx_add).
// Two deposit paths, both exact forms of that formula:
//   common: on every axis the old and the new position round to the same
//     node (TSC) / stay in the same cell (CIC), so the union of the two
//     supports is 3 (TSC) / 2 (CIC) nodes and DS has closed per-node forms
//     in the displacement D (no cancellation in FP32); 54 (TSC) / 12 (CIC)
//     shared atomics, no branches;
//   queued: the rest (a few percent of particles) wait in a shared queue and
//     are deposited with the general 4-node window by full warps, so the
//     rare case costs no divergence in the common loop.
// The shared tiles use an odd row pitch so that the 32 banks spread over
// neighbouring rows.
#include "pic_internal.cuh"

#include <cmath>

namespace pic {

constexpr int kHoleCap = 512;

template <int LX_, int LY_, int LZ_>
struct Tile {
    static constexpr int LX = LX_, LY = LY_, LZ = LZ_;
    static constexpr int TX = LX + 4;  // x: one guard below, three above (16-byte rows)
    static constexpr int TY = LY + 3;  // y, z: one guard below, two above
    static constexpr int TZ = LZ + 3;
    static constexpr int PX = TX + 1;  // odd shared-memory row pitch
    static constexpr int N = PX * TY * TZ;  // shared floats per component
    static constexpr int S = LX * LY * LZ;
};

// ------------------------------------------------------------ shape factors

// TSC (quadratic spline, Hockney & Eastwood) at distance d, branch-free.
__device__ __forceinline__ float tsc_S(float d)
{
    float a = fabsf(d);
    float t = fmaxf(1.5f - a, 0.0f);
    return a <= 0.5f ? 0.75f - a * a : 0.5f * t * t;
}

// S(d0 + D) - S(d0) for TSC; when both ends lie on one spline piece the
// difference is factored through D so it keeps FP32 relative accuracy.
__device__ __forceinline__ float tsc_dS(float d0, float D)
{
    float d1 = d0 + D;
    float a0 = fabsf(d0), a1 = fabsf(d1);
    int p0 = a0 <= 0.5f ? 0 : (a0 < 1.5f ? 1 : 2);
    int p1 = a1 <= 0.5f ? 0 : (a1 < 1.5f ? 1 : 2);
    float s = d0 >= 0.0f ? 1.0f : -1.0f;  // |D| < 1/2: both outer ends share the sign
    float centre = -D * (d0 + d1);
    float outer = -0.5f * s * D * (3.0f - s * (d0 + d1));
    float general = tsc_S(d1) - tsc_S(d0);
    float same = p0 == 0 ? centre : (p0 == 1 ? outer : 0.0f);
    return p0 == p1 ? same : general;
}

__device__ __forceinline__ float cic_S(float d) { return fmaxf(0.0f, 1.0f - fabsf(d)); }

__device__ __forceinline__ float cic_dS(float d0, float D)
{
    float d1 = d0 + D;
    bool same = fabsf(d0) < 1.0f && fabsf(d1) < 1.0f && ((d0 >= 0.0f) == (d1 >= 0.0f));
    float f = d0 >= 0.0f ? -D : D;
    return same ? f : cic_S(d1) - cic_S(d0);
}

// Gather weights along one axis for a particle at offset o in [0,1) of its
// cell; the tile coordinate of the particle's cell is l + 1.  "i" = field
// sampled at integer nodes along this axis, "h" = at half nodes.  For the
// integer nodes the weights are also the particle's shape S0 at the nodes
// a-1, a, a+1 (TSC, a = round(o)) or 0, 1 (CIC): the deposit reuses them.
template <int SHAPE>
struct AxisW {
    static constexpr int NW = SHAPE == 2 ? 3 : 2;
    int bi, bh;  // tile index of the first node
    float wi[NW], wh[NW];
    float di;    // TSC: o - a
    __device__ __forceinline__ AxisW(int l, float o)
    {
        if (SHAPE == 2) {
            bool up = o >= 0.5f;
            di = up ? o - 1.0f : o;
            bi = l + (up ? 1 : 0);
            float a = 0.5f - di, c = 0.5f + di;
            wi[0] = 0.5f * a * a;
            wi[1] = 0.75f - di * di;
            wi[2] = 0.5f * c * c;
            float dh = o - 0.5f;
            bh = l;
            float ah = 0.5f - dh, ch = 0.5f + dh;
            wh[0] = 0.5f * ah * ah;
            wh[1] = 0.75f - dh * dh;
            wh[2] = 0.5f * ch * ch;
        } else {
            di = o;
            bi = l + 1;
            wi[0] = 1.0f - o;
            wi[1] = o;
            bool up = o >= 0.5f;
            float dh = up ? o - 0.5f : o + 0.5f;
            bh = l + (up ? 1 : 0);
            wh[0] = 1.0f - dh;
            wh[1] = dh;
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

// Esirkepov transverse factor S0e S0f + (DSe S0f + S0e DSf)/2 + DSe DSf / 3.
__device__ __forceinline__ float esk_T(float s0e, float dse, float s0f, float dsf)
{
    return fmaf(s0e, s0f, fmaf(0.5f, fmaf(dse, s0f, s0e * dsf), (1.0f / 3.0f) * dse * dsf));
}

// ------------------------------------------------------------ fixed-point J tile
//
// The shared J tile accumulates in integers: shared-memory int32 atomics are
// native and combine lanes that hit one address, where FP32 shared atomics
// are a compare-and-swap loop that serialises them.  A contribution v (already
// multiplied by the tile scale s) is split into hi = floor(v) and lo =
// round((v - hi) 2^m), added to two int32 accumulators; the tile value is
// (hi_sum 2^m + lo_sum) / (s 2^m).  The scale comes from a bound on every
// contribution (|P| <= |D| < 1/2, |T| <= 1, |coef w| <= cbound) and on the
// number of contributions per node (the particles of the supercell), so no
// accumulator can overflow; the resolution is about 2^-42 of the bound.
// Conversions use the 1.5 * 2^23 magic-number add (|h|, lo < 2^22).
struct FxScale {
    float s;      // multiply a contribution by s to get hi units
    float two_m;  // 2^m: lo units per hi unit
    float inv;    // 1 / (s 2^m): back to current density
};

__device__ __forceinline__ int magic_int(float x)
{
    return __float_as_int(x + 12582912.0f) - 0x4B400000;
}

__device__ __forceinline__ void fx_add(int* hi, int* lo, float v, float two_m)
{
    const float h = floorf(v);
    const float l = (v - h) * two_m;
    atomicAdd(hi, magic_int(h));
    atomicAdd(lo, magic_int(l));
}

__device__ __forceinline__ FxScale fx_scale(int ntot, float bound)
{
    const int lg = ntot > 1 ? 32 - __clz(ntot - 1) : 0;  // ceil(log2 ntot)
    const int m = min(22, 30 - lg);
    const int hb = min(21, 30 - lg);
    int e = 0;
    if (bound > 0.0f)
        frexpf(bound, &e);  // bound <= 2^e
    FxScale f;
    f.s = ldexpf(1.0f, hb - e);
    f.two_m = ldexpf(1.0f, m);
    f.inv = ldexpf(1.0f, e - hb - m);
    return f;
}

// Deposit the three current components on a window of M nodes per axis
// (M-1 half nodes along the current's own axis); node 0 of axis d sits at
// tile index b[d].  cx..cz carry q w / (V dt) h_d and the tile scale.
template <int M, int PX, int TY, int NJ>
__device__ __forceinline__ void deposit_window(int* sJh, int* sJl, const int b[3], const float* S0x,
                                               const float* S0y, const float* S0z, const float* DSx,
                                               const float* DSy, const float* DSz, float cx, float cy,
                                               float cz, float two_m)
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
            for (int j = 0; j < M; ++j) {
                const float T = cx * esk_T(S0y[j], DSy[j], S0z[k], DSz[k]);
                const int row = (b[2] + k) * PY + (b[1] + j) * PX + b[0];
#pragma unroll
                for (int i = 0; i < M - 1; ++i)
                    fx_add(sJh + row + i, sJl + row + i, P[i] * T, two_m);
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
            for (int i = 0; i < M; ++i) {
                const float T = cy * esk_T(S0z[k], DSz[k], S0x[i], DSx[i]);
                const int col = NJ + (b[2] + k) * PY + b[1] * PX + (b[0] + i);
#pragma unroll
                for (int j = 0; j < M - 1; ++j)
                    fx_add(sJh + col + j * PX, sJl + col + j * PX, P[j] * T, two_m);
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
            for (int i = 0; i < M; ++i) {
                const float T = cz * esk_T(S0x[i], DSx[i], S0y[j], DSy[j]);
                const int col = 2 * NJ + b[2] * PY + (b[1] + j) * PX + (b[0] + i);
#pragma unroll
                for (int k = 0; k < M - 1; ++k)
                    fx_add(sJh + col + k * PY, sJl + col + k * PY, P[k] * T, two_m);
            }
    }
}

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

// Exclusive prefix sum of cnt[0..K) into off[0..K) by the whole block.
template <int NT>
__device__ void block_exclusive_scan_counts(const int* cnt, int* off, int K, int* s_warp)
{
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int per = (K + NT - 1) / NT;
    const int b0 = tid * per;
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
    if (lane == 31)
        s_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int t = lane < NT / 32 ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o)
                t += y;
        }
        if (lane < NT / 32)
            s_warp[lane] = t;
    }
    __syncthreads();
    int run = x - local + (wid > 0 ? s_warp[wid - 1] : 0);
    for (int i = 0; i < per; ++i)
        if (b0 + i < K) {
            off[b0 + i] = run;
            run += cnt[b0 + i];
        }
}

// ------------------------------------------------------------ shared state

// Particles of one chunk of a frame list, staged in shared memory in list
// order, plus their counting-sort permutation by nearest node.
template <int C>
struct Stage {
    int cell[C];
    float o[3][C];
    float u[3][C];
    float w[C];
    int pid[C];   // particle ids (only when tracked)
    int kr[C];    // key << 16 | rank within key
    int perm[C];  // sorted position -> chunk position
};

// Particles whose move needs the general 4-node window.
template <int C>
struct DepositQueue {
    int l[C];        // packed local cell coordinates lx | ly << 8 | lz << 16
    float o[3][C];   // old in-cell offsets
    float D[3][C];   // displacement in cells
    float w[C];      // weight
};

template <class T, int SHAPE, int C>
__device__ __forceinline__ void deposit_queued(int* sJh, int* sJl, const DepositQueue<C>& q, int e,
                                               const float jc[3], const FxScale& fx)
{
    const int l = q.l[e];
    float S0[3][4], DS[3][4];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float o = q.o[a][e], D = q.D[a][e];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float d0 = o - (float)(k - 1);
            S0[a][k] = SHAPE == 2 ? tsc_S(d0) : cic_S(d0);
            DS[a][k] = SHAPE == 2 ? tsc_dS(d0, D) : cic_dS(d0, D);
        }
    }
    const int b[3] = {l & 0xff, (l >> 8) & 0xff, l >> 16};  // node l-1 sits at tile index l
    const float w = q.w[e] * fx.s;
    deposit_window<4, T::PX, T::TY, T::N>(sJh, sJl, b, S0[0], S0[1], S0[2], DS[0], DS[1], DS[2],
                                          jc[0] * w, jc[1] * w, jc[2] * w, fx.two_m);
}

template <class T, int SHAPE>
struct Keys {
    static constexpr int K = SHAPE == 2 ? (T::LX + 1) * (T::LY + 1) * (T::LZ + 1) : T::S;
};

template <class T>
constexpr int max_keys()
{
    return (T::LX + 1) * (T::LY + 1) * (T::LZ + 1);
}

template <class T, int NT>
struct SharedState {
    static constexpr int C = 2 * NT;
    Stage<C> st;
    DepositQueue<C> q;
    int hist[max_keys<T>()];
    int off[max_keys<T>()];
    int holes[kHoleCap];
    int src[kHoleCap];
    int warp[32];
    int item, any, nq, nholes, nhead, nsrc;
    FxScale fx;
};

// ------------------------------------------------------------ one particle

template <class T, int SHAPE, int C>
__device__ __forceinline__ void push_one(const StepDev& d, const SpeciesDev& sp, int s, const BoxDev& bx,
                                         int scx, int scy, int scz, const float* sF, int* sJh, int* sJl,
                                         Stage<C>& st, DepositQueue<C>& q, int& s_nq, int& s_nholes,
                                         int* s_holes, const FxScale& fx, int j, int p,
                                         unsigned& my_status)
{
    constexpr int LX = T::LX, LY = T::LY, LZ = T::LZ, N = T::N, PX = T::PX, TY = T::TY;
    constexpr int NW = SHAPE == 2 ? 3 : 2;
    const int cell = st.cell[j];
    const float ox = st.o[0][j], oy = st.o[1][j], oz = st.o[2][j];
    float ux = st.u[0][j], uy = st.u[1][j], uz = st.u[2][j];
    const float w = st.w[j];
    const int lx = cell % LX;
    const int ly = (cell / LX) % LY;
    const int lz = cell / (LX * LY);

    // gather (Sec. 4: product of 1D weights at each Yee position)
    AxisW<SHAPE> ax(lx, ox), ay(ly, oy), az(lz, oz);
    const float Ex = gather_comp<NW, PX, TY>(sF + 0 * N, ax.bh, ay.bi, az.bi, ax.wh, ay.wi, az.wi);
    const float Ey = gather_comp<NW, PX, TY>(sF + 1 * N, ax.bi, ay.bh, az.bi, ax.wi, ay.wh, az.wi);
    const float Ez = gather_comp<NW, PX, TY>(sF + 2 * N, ax.bi, ay.bi, az.bh, ax.wi, ay.wi, az.wh);
    const float Bx = gather_comp<NW, PX, TY>(sF + 3 * N, ax.bi, ay.bh, az.bh, ax.wi, ay.wh, az.wh);
    const float By = gather_comp<NW, PX, TY>(sF + 4 * N, ax.bh, ay.bi, az.bh, ax.wh, ay.wi, az.wh);
    const float Bz = gather_comp<NW, PX, TY>(sF + 5 * N, ax.bh, ay.bh, az.bi, ax.wh, ay.wh, az.wi);

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

    // Esirkepov deposition
    bool common;
    if (SHAPE == 2)
        common = ((ox >= 0.5f) == (x1 >= 0.5f)) && ((oy >= 0.5f) == (y1 >= 0.5f)) &&
                 ((oz >= 0.5f) == (z1 >= 0.5f));
    else
        common = x1 >= 0.0f && x1 < 1.0f && y1 >= 0.0f && y1 < 1.0f && z1 >= 0.0f && z1 < 1.0f;
    if (common) {
        float DSx[NW], DSy[NW], DSz[NW];
        if (SHAPE == 2) {
            // nodes a-1, a, a+1 with delta = o - a (d1 = d0 + D):
            // DS = -D/2 (1 - d0 - d1), -D (d0 + d1), D/2 (1 + d0 + d1)
            const float Ds[3] = {Dx, Dy, Dz};
            const float dl[3] = {ax.di, ay.di, az.di};
            float* out[3] = {DSx, DSy, DSz};
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float sum = 2.0f * dl[a] + Ds[a];
                out[a][0] = -0.5f * Ds[a] * (1.0f - sum);
                out[a][1] = -Ds[a] * sum;
                out[a][2] = 0.5f * Ds[a] * (1.0f + sum);
            }
        } else {
            DSx[0] = -Dx;
            DSx[1] = Dx;
            DSy[0] = -Dy;
            DSy[1] = Dy;
            DSz[0] = -Dz;
            DSz[1] = Dz;
        }
        const int b[3] = {ax.bi, ay.bi, az.bi};
        const float ws = w * fx.s;
        deposit_window<NW, PX, TY, N>(sJh, sJl, b, ax.wi, ay.wi, az.wi, DSx, DSy, DSz,
                                      sp.jcoef[0] * ws, sp.jcoef[1] * ws, sp.jcoef[2] * ws, fx.two_m);
    } else {
        const int e = atomicAdd(&s_nq, 1);  // < C: one entry per particle of the chunk
        q.l[e] = lx | (ly << 8) | (lz << 16);
        q.o[0][e] = ox;
        q.o[1][e] = oy;
        q.o[2][e] = oz;
        q.D[0][e] = Dx;
        q.D[1][e] = Dy;
        q.D[2][e] = Dz;
        q.w[e] = w;
    }

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
        st.cell[j] = nlx + LX * (nly + LY * nlz);
        st.o[0][j] = nox;
        st.o[1][j] = noy;
        st.o[2][j] = noz;
        st.u[0][j] = ux;
        st.u[1][j] = uy;
        st.u[2][j] = uz;
    } else {
        // leaves the supercell: into the move buffer, towards the neighbour
        // supercell (periodic within the box)
        int tsx = scx + dsx, tsy = scy + dsy, tsz = scz + dsz;
        tsx += tsx < 0 ? bx.nscx : (tsx >= bx.nscx ? -bx.nscx : 0);
        tsy += tsy < 0 ? bx.nscy : (tsy >= bx.nscy ? -bx.nscy : 0);
        tsz += tsz < 0 ? bx.nscz : (tsz >= bx.nscz ? -bx.nscz : 0);
        const int dest_sc = bx.sc_base + (tsz * bx.nscy + tsy) * bx.nscx + tsx;
        const int dest_cell = (nlx - dsx * LX) + LX * ((nly - dsy * LY) + LY * (nlz - dsz * LZ));
        const int destL = s * d.nsc + dest_sc;
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
                d.mv_pid[m] = st.pid[j];
        } else {
            my_status |= ST_CAPACITY;
        }
        st.cell[j] = -1;
        const int h = atomicAdd(&s_nholes, 1);
        if (h < kHoleCap)
            s_holes[h] = p;
    }
}

// ------------------------------------------------------------ one frame list

template <class T, int SHAPE, int NT>
__device__ __forceinline__ void push_list(const StepDev& d, const SpeciesDev& sp, int s, int g,
                                          const BoxDev& bx, int scx, int scy, int scz,
                                          const float* sF, int* sJh, int* sJl,
                                          SharedState<T, NT>& sh, unsigned& my_status)
{
    constexpr int LX = T::LX, LY = T::LY, S = T::S;
    constexpr int C = SharedState<T, NT>::C;
    constexpr int K = Keys<T, SHAPE>::K;
    const int tid = threadIdx.x;
    const int L = s * d.nsc + g;
    const int n = d.count[L];
    const int* ft = d.ftab + d.foff[L];
    for (int base = 0; base < n; base += C) {
        const int cn = min(C, n - base);
        for (int k = tid; k < K; k += NT)
            sh.hist[k] = 0;
        __syncthreads();
        // stage the chunk (coalesced), key = nearest node (TSC) / cell (CIC)
        for (int j = tid; j < cn; j += NT) {
            const int p = base + j;
            const int64_t idx = (int64_t)ft[p >> d.log2S] * S + (p & (S - 1));
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
        block_exclusive_scan_counts<NT>(sh.hist, sh.off, K, sh.warp);
        __syncthreads();
        for (int j = tid; j < cn; j += NT) {
            const int kr = sh.st.kr[j];
            sh.st.perm[sh.off[kr >> 16] + (kr & 0xffff)] = j;
        }
        __syncthreads();
        // push in sorted order: neighbouring lanes share cells
        for (int sidx = tid; sidx < cn; sidx += NT) {
            const int j = sh.st.perm[sidx];
            push_one<T, SHAPE, C>(d, sp, s, bx, scx, scy, scz, sF, sJh, sJl, sh.st, sh.q, sh.nq,
                                  sh.nholes, sh.holes, sh.fx, j, base + j, my_status);
        }
        __syncthreads();
        // queued moves with the general window, then write the chunk back
        const int nq = sh.nq;
        for (int e = tid; e < nq; e += NT)
            deposit_queued<T, SHAPE, C>(sJh, sJl, sh.q, e, sp.jcoef, sh.fx);
        for (int j = tid; j < cn; j += NT) {
            const int p = base + j;
            const int64_t idx = (int64_t)ft[p >> d.log2S] * S + (p & (S - 1));
            const int cell = sh.st.cell[j];
            d.cell[idx] = cell;
            if (cell >= 0) {
                d.ox[idx] = sh.st.o[0][j];
                d.oy[idx] = sh.st.o[1][j];
                d.oz[idx] = sh.st.o[2][j];
                d.ux[idx] = sh.st.u[0][j];
                d.uy[idx] = sh.st.u[1][j];
                d.uz[idx] = sh.st.u[2][j];
            }
        }
        __syncthreads();
        if (tid == 0)
            sh.nq = 0;
    }
}

// Fill the holes the leavers left below n - nholes with the survivors above.
template <class T, int NT>
__device__ __forceinline__ void compact_list(const StepDev& d, int L, int n, int nh, const int* s_holes,
                                             int* s_src, int& s_nhead, int& s_nsrc)
{
    constexpr int S = T::S;
    const int tid = threadIdx.x;
    const int nstay = n - nh;
    const int* ft = d.ftab + d.foff[L];
    auto gidx = [&](int slot) -> int64_t { return (int64_t)ft[slot >> d.log2S] * S + (slot & (S - 1)); };
    auto move_particle = [&](int from, int to) {
        const int64_t a = gidx(from), b = gidx(to);
        d.cell[b] = d.cell[a];
        d.ox[b] = d.ox[a];
        d.oy[b] = d.oy[a];
        d.oz[b] = d.oz[a];
        d.ux[b] = d.ux[a];
        d.uy[b] = d.uy[a];
        d.uz[b] = d.uz[a];
        d.w[b] = d.w[a];
        if (d.pid)
            d.pid[b] = d.pid[a];
    };
    if (nh <= kHoleCap) {
        if (tid == 0) {
            s_nhead = 0;
            s_nsrc = 0;
        }
        __syncthreads();
        // survivors in the tail [nstay, n)
        for (int t = tid; t < nh; t += NT) {
            const int slot = nstay + t;
            if (d.cell[gidx(slot)] != -1)
                s_src[atomicAdd(&s_nsrc, 1)] = slot;
        }
        __syncthreads();
        // holes in the head [0, nstay): as many as tail survivors
        for (int t = tid; t < nh; t += NT) {
            const int hs = s_holes[t];
            if (hs < nstay)
                move_particle(s_src[atomicAdd(&s_nhead, 1)], hs);
        }
    } else if (tid < 32) {
        // many leavers: warp-wide two-pointer scan over the list
        const int lane = tid;
        int a = 0, b = nstay, ha = 0, hb = 0;
        unsigned ma = 0, mb = 0;
        while (true) {
            while (ma == 0 && a < nstay) {
                const int slot = a + lane;
                ma = __ballot_sync(0xffffffffu, slot < nstay && d.cell[gidx(slot)] == -1);
                ha = a;
                a += 32;
            }
            while (mb == 0 && b < n) {
                const int slot = b + lane;
                mb = __ballot_sync(0xffffffffu, slot < n && d.cell[gidx(slot)] != -1);
                hb = b;
                b += 32;
            }
            if (ma == 0 || mb == 0)
                break;
            const int k = min(__popc(ma), __popc(mb));
            if (lane < k) {  // lane r moves the r-th survivor into the r-th hole
                unsigned xa = ma, xb = mb;
                for (int r = 0; r < lane; ++r) {
                    xa &= xa - 1;
                    xb &= xb - 1;
                }
                move_particle(hb + __ffs(xb) - 1, ha + __ffs(xa) - 1);
            }
            __syncwarp();
            for (int r = 0; r < k; ++r) {
                ma &= ma - 1;
                mb &= mb - 1;
            }
        }
    }
}

// ------------------------------------------------------------ the kernel

template <class T, int NT>
__global__ void __launch_bounds__(NT, 768 / NT) k_push_deposit(const StepDev d)
{
    constexpr int TX = T::TX, TY = T::TY, TZ = T::TZ, PX = T::PX, N = T::N;
    constexpr int LX = T::LX, LY = T::LY, LZ = T::LZ;
    extern __shared__ __align__(16) float smem[];
    // layout (dyn_smem): [6N field floats][3N hi ints][3N lo ints][SharedState]
    float* sF = smem;                                     // [6][TZ][TY][PX]: Ex Ey Ez Bx By Bz
    int* sJh = reinterpret_cast<int*>(smem + 6 * N);      // [3][TZ][TY][PX] hi words
    int* sJl = sJh + 3 * N;                               // [3][TZ][TY][PX] lo words
    SharedState<T, NT>& sh = *reinterpret_cast<SharedState<T, NT>*>(sJl + 3 * N);

    const int tid = threadIdx.x;
    unsigned my_status = 0;

    for (;;) {
        if (tid == 0)
            sh.item = atomicAdd(d.work_counter, 1);
        __syncthreads();
        const int item = sh.item;
        if (item >= d.nsc)
            break;
        const int g = d.items[item];
        const BoxDev bx = d.boxes[d.sc_box[g]];
        const int loc = g - bx.sc_base;
        const int scx = loc % bx.nscx;
        const int scy = (loc / bx.nscx) % bx.nscy;
        const int scz = loc / (bx.nscx * bx.nscy);

        if (tid == 0) {
            int ntot = 0;
            float bound = 0.0f;
            for (int s = 0; s < d.nspecies; ++s) {
                const int c = d.count[s * d.nsc + g];
                if (d.sp[s].mobile && c > 0) {
                    ntot += c;
                    bound = fmaxf(bound, 0.5f * d.sp[s].cbound);
                }
            }
            sh.any = ntot;
            sh.fx = fx_scale(ntot, bound);
        }
        __syncthreads();
        if (sh.any == 0) {
            __syncthreads();  // item / any are rewritten next round
            continue;
        }

        // ---- 1. stage the E/B tile, zero the J tile
        const int64_t pcell = padded_cells(bx);
        const int64_t start = ((int64_t)(scz * LZ) * bx.py + scy * LY) * bx.px + scx * LX;
        constexpr int ROW4 = TX / 4;
        constexpr int NV = 6 * TZ * TY * ROW4;
        for (int v = tid; v < NV; v += NT) {
            const int r4 = v % ROW4;
            const int row = v / ROW4;  // (c * TZ + tz) * TY + ty
            const int ty = row % TY;
            const int tz = (row / TY) % TZ;
            const int c = row / (TY * TZ);
            const float* base = (c < 3 ? bx.E : bx.B) + (c % 3) * pcell;
            const float4 val = __ldg(reinterpret_cast<const float4*>(
                                         base + start + ((int64_t)tz * bx.py + ty) * bx.px) + r4);
            float* dst = sF + row * PX + 4 * r4;
            dst[0] = val.x;
            dst[1] = val.y;
            dst[2] = val.z;
            dst[3] = val.w;
        }
        for (int v = tid; v < 6 * N; v += NT)
            sJh[v] = 0;  // hi and lo words are contiguous
        if (tid == 0)
            sh.nq = 0;
        __syncthreads();

        // ---- 2. particles of every mobile species, 3. compaction
        for (int s = 0; s < d.nspecies; ++s) {
            const SpeciesDev sp = d.sp[s];
            const int L = s * d.nsc + g;
            const int n = d.count[L];
            if (!sp.mobile || n == 0)
                continue;
            if (tid == 0)
                sh.nholes = 0;
            __syncthreads();
            if (sp.shape == 2)
                push_list<T, 2, NT>(d, sp, s, g, bx, scx, scy, scz, sF, sJh, sJl, sh, my_status);
            else
                push_list<T, 1, NT>(d, sp, s, g, bx, scx, scy, scz, sF, sJh, sJl, sh, my_status);
            __syncthreads();
            const int nh = sh.nholes;
            if (nh > 0) {
                compact_list<T, NT>(d, L, n, nh, sh.holes, sh.src, sh.nhead, sh.nsrc);
                __syncthreads();
                if (tid == 0)
                    d.count[L] = n - nh;
            }
            __syncthreads();
        }

        // ---- 4. add the J tile to global J
        const FxScale fx = sh.fx;
        constexpr int NJ4 = 3 * TZ * TY * ROW4;
        for (int v = tid; v < NJ4; v += NT) {
            const int r4 = v % ROW4;
            const int row = v / ROW4;
            const int e = row * PX + 4 * r4;
            float val[4];
            bool any = false;
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int hi = sJh[e + t], lo = sJl[e + t];
                any |= (hi | lo) != 0;
                val[t] = fmaf((float)hi, fx.two_m, (float)lo) * fx.inv;
            }
            if (any) {
                const int ty = row % TY;
                const int tz = (row / TY) % TZ;
                const int c = row / (TY * TZ);
                float* dst = bx.J + c * pcell + start + ((int64_t)tz * bx.py + ty) * bx.px + 4 * r4;
                atomicAdd(reinterpret_cast<float4*>(dst), make_float4(val[0], val[1], val[2], val[3]));
            }
        }
        __syncthreads();
    }
    if (my_status)
        atomicOr(d.status, my_status);
}

// ------------------------------------------------------------ dispatch

template <class T, int NT>
static size_t dyn_smem()
{
    // field tile (6 N floats) + fixed-point current tile (3 N hi + 3 N lo ints) + shared state
    return sizeof(float) * 12 * T::N + sizeof(SharedState<T, NT>);
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

#define PIC_PUSH_CASES(X)  \
    X(4, 4, 4, 64)         \
    X(4, 4, 4, 128)        \
    X(8, 4, 4, 128)        \
    X(8, 8, 4, 128)        \
    X(8, 8, 4, 256)        \
    X(8, 8, 8, 256)

size_t push_smem_bytes(int LX, int LY, int LZ, int threads)
{
#define X(a, b, c, t)                                          \
    if (LX == a && LY == b && LZ == c && threads == t)         \
        return dyn_smem<Tile<a, b, c>, t>();
    PIC_PUSH_CASES(X)
#undef X
    return 0;
}

int push_supported(int LX, int LY, int LZ, int threads)
{
#define X(a, b, c, t) if (LX == a && LY == b && LZ == c && threads == t) return 1;
    PIC_PUSH_CASES(X)
#undef X
    return 0;
}

cudaError_t configure_push(int LX, int LY, int LZ, int threads, int* per_sm)
{
#define X(a, b, c, t)                                          \
    if (LX == a && LY == b && LZ == c && threads == t)         \
        return configure_one<Tile<a, b, c>, t>(per_sm);
    PIC_PUSH_CASES(X)
#undef X
    return cudaErrorInvalidValue;
}

cudaError_t launch_push_deposit(const StepDev& d, int threads, int grid, cudaStream_t st)
{
#define X(a, b, c, t)                                          \
    if (d.LX == a && d.LY == b && d.LZ == c && threads == t)   \
        return launch_one<Tile<a, b, c>, t>(d, grid, st);
    PIC_PUSH_CASES(X)
#undef X
    return cudaErrorInvalidValue;
}

}  // namespace pic
