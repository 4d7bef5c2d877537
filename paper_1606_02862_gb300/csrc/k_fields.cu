// k_fields.cu -- Yee FDTD update (Yee 1966, the "Yee field solver" of Sec. 4)
// for the mixed form's guard-padded FP32 fields, field import/export, and
// the FP64 diagnostics reductions.
//
// Staggering: Ex(i+1/2,j,k) Ey(i,j+1/2,k) Ez(i,j,k+1/2), Bx(i,j+1/2,k+1/2)
// By(i+1/2,j,k+1/2) Bz(i+1/2,j+1/2,k); J with E.  One step of the field
// half of the cycle:
//   B^{n+1/2} = B^n - dt/2 curl E^n
//   E^{n+1}   = E^n + dt (curl B^{n+1/2} - J^{n+1/2})
//   B^{n+1}   = B^{n+1/2} - dt/2 curl E^{n+1}
// Every kernel writes each updated interior value also into its periodic
// guard images, so the next kernel (and the next push's tile loads) read
// guards without a separate exchange.  The E kernel folds the J guard
// images (deposits that spilled over the periodic seam) into the current of
// each interior cell as it reads it; J itself stays as deposited (the step
// zeroes it before the push, and a read of J folds the same way).
//
// One launch covers all boxes: blocks of 32 x 8 cells in x-y, each thread
// kYeeZ cells along z, box found from a per-box block offset table.
#include "pic_internal.cuh"
#include "tma.cuh"

#include <algorithm>
#include <cmath>

namespace pic {

constexpr int kYeeZ = kYeeCellsZ;  // box edges are multiples of the supercell edge, >= 4

struct YeeArgs {
    const BoxDev* boxes;
    const int* blk_off;  // [nboxes + 1]
    int nboxes;
    float tau;           // dt/2 for the B halves, dt for E
    float ih[3];         // 1 / h_d
    const long long* step_no;
    double dt_d;
    double dx_d[3];
};

__device__ __forceinline__ int find_box(const int* off, int n, int blk)
{
    int lo = 0, hi = n;  // off[lo] <= blk < off[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (off[mid] <= blk)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

struct CellAt {
    int x, y, z;
    bool ok;
};

__device__ __forceinline__ CellAt yee_cell(const YeeArgs& a, const BoxDev*& bp)
{
    const int box = find_box(a.blk_off, a.nboxes, blockIdx.x);
    bp = a.boxes + box;  // fields read through the pointer as used, not copied
    const BoxDev& b = *bp;
    const int local = blockIdx.x - a.blk_off[box];
    const int nbx = (b.nx + 31) >> 5, nby = (b.ny + 7) >> 3;
    CellAt c;
    c.x = (local % nbx) * 32 + threadIdx.x;
    c.y = ((local / nbx) % nby) * 8 + threadIdx.y;
    c.z = local / (nbx * nby);
    c.ok = c.x < b.nx && c.y < b.ny;
    return c;
}

// Periodic images of an interior coordinate v in [0, n) inside the padded
// range [-lo, n + hi): v itself, and v + n when v < hi or v - n when
// v >= n - lo.  Boxes are at least lo + hi cells long (4 for CIC/TSC
// guards, 8 with the PCS guards), so at most one of the two applies.
// Returns the count (1 or 2), [0] = v.
__device__ __forceinline__ int images(int v, int n, int lo, int hi, int* out)
{
    out[0] = v;
    if (v < hi) {
        out[1] = v + n;
        return 2;
    }
    if (v >= n - lo) {
        out[1] = v - n;
        return 2;
    }
    return 1;
}

__device__ __forceinline__ int images_x(const BoxDev& b, int v, int* out)
{
    return images(v, b.nx, b.gx, b.px - b.nx - b.gx, out);
}
__device__ __forceinline__ int images_y(const BoxDev& b, int v, int* out)
{
    return images(v, b.ny, b.gy, b.py - b.ny - b.gy, out);
}
__device__ __forceinline__ int images_z(const BoxDev& b, int v, int* out)
{
    return images(v, b.nz, b.gz, b.pz - b.nz - b.gz, out);
}

__device__ __forceinline__ void store_with_images(const BoxDev& b, float* F, const CellAt& c,
                                                  float v)
{
    int ix[2], iy[2], iz[2];
    int nx = images_x(b, c.x, ix), ny = images_y(b, c.y, iy), nz = images_z(b, c.z, iz);
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i)
                F[padded_index(b, ix[i], iy[j], iz[k])] = v;
}

// The Yee kernels take the guard layout as a template constant (G = 1:
// CIC/TSC contexts, 2: PCS), so that the image arithmetic of every cell is
// immediate.
template <int G>
struct GuardsOf {
    static constexpr int hx = G == 1 ? 3 : 6, hyz = G == 1 ? 2 : 3;
};

template <int G>
__device__ __forceinline__ int64_t pidx(const BoxDev& b, int x, int y, int z)
{
    return ((int64_t)(z + G) * b.py + (y + G)) * b.px + (x + G);
}

template <int G>
__device__ __forceinline__ void store_images_g(const BoxDev& b, float* F, const CellAt& c, float v)
{
    int ix[2], iy[2], iz[2];
    const int nx = images(c.x, b.nx, G, GuardsOf<G>::hx, ix);
    const int ny = images(c.y, b.ny, G, GuardsOf<G>::hyz, iy);
    const int nz = images(c.z, b.nz, G, GuardsOf<G>::hyz, iz);
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i)
                F[pidx<G>(b, ix[i], iy[j], iz[k])] = v;
}

// Each thread updates kYeeZ cells stacked in z: all loads first, then the
// arithmetic and the stores, so that a warp keeps kYeeZ times the bytes in
// flight (the update is bound by DRAM latency with one cell per thread).
template <int G>
__global__ void __launch_bounds__(256) k_yee_b(const YeeArgs a)
{
    const BoxDev* bp;
    CellAt c = yee_cell(a, bp);
    if (!c.ok)
        return;
    const BoxDev& b = *bp;
    const int64_t pc = padded_cells(b);
    const int64_t sx = 1, sy = b.px, sz = (int64_t)b.px * b.py;
    const float* __restrict__ Ex = b.E;
    const float* __restrict__ Ey = b.E + pc;
    const float* __restrict__ Ez = b.E + 2 * pc;
    float* __restrict__ Bx = b.B;
    float* __restrict__ By = b.B + pc;
    float* __restrict__ Bz = b.B + 2 * pc;
    const int z0 = c.z * kYeeZ;
    float cx[kYeeZ], cy[kYeeZ], cz[kYeeZ], bx[kYeeZ], by[kYeeZ], bz[kYeeZ];
    // Ex, Ey one plane up are the next cell's own values (the thread's cells
    // are stacked in z): kYeeZ + 1 planes of them, loaded once
    float exs[kYeeZ + 1], eys[kYeeZ + 1];
#pragma unroll
    for (int q = 0; q <= kYeeZ; ++q) {
        const int64_t i = pidx<G>(b, c.x, c.y, z0 + q);
        exs[q] = __ldg(Ex + i);
        eys[q] = __ldg(Ey + i);
    }
#pragma unroll
    for (int q = 0; q < kYeeZ; ++q) {
        const int64_t i = pidx<G>(b, c.x, c.y, z0 + q);
        const float ex = exs[q], ey = eys[q], ez = __ldg(Ez + i);
        cx[q] = (__ldg(Ez + i + sy) - ez) * a.ih[1] - (eys[q + 1] - ey) * a.ih[2];
        cy[q] = (exs[q + 1] - ex) * a.ih[2] - (__ldg(Ez + i + sx) - ez) * a.ih[0];
        cz[q] = (__ldg(Ey + i + sx) - ey) * a.ih[0] - (__ldg(Ex + i + sy) - ex) * a.ih[1];
        bx[q] = Bx[i];
        by[q] = By[i];
        bz[q] = Bz[i];
    }
#pragma unroll
    for (int q = 0; q < kYeeZ; ++q) {
        c.z = z0 + q;
        store_images_g<G>(b, Bx, c, bx[q] - a.tau * cx[q]);
        store_images_g<G>(b, By, c, by[q] - a.tau * cy[q]);
        store_images_g<G>(b, Bz, c, bz[q] - a.tau * cz[q]);
    }
}

// Laser antenna: adds the sheet current at the Ex positions
// (x+1/2, ant_j, z) of every box with an antenna into J, at the time of this
// step's current, t = (n + 1/2) dt, n = steps taken before it (step_no was
// advanced earlier in the step).  Runs before the E update, which folds it
// in with the deposits.  FP64 throughout: omega t reaches thousands of
// radians.  One thread per (box, x, z), grid-stride.
__device__ __forceinline__ float antenna_current(const YeeArgs& a, const BoxDev& b, int x, int z)
{
    const OpenYDev& o = b.oy;
    const double t = ((double)(*a.step_no) - 0.5) * a.dt_d;
    const double T = o.ant_tau > 0.0 ? exp(-((t - o.ant_t0) / o.ant_tau) * ((t - o.ant_t0) / o.ant_tau)) : 1.0;
    double G = 1.0;
    if (o.ant_w0 > 0.0) {
        const double px = ((double)x + 0.5) * a.dx_d[0] - o.ant_xc;
        const double pz = (double)z * a.dx_d[2] - o.ant_zc;
        G = exp(-(px * px + pz * pz) / (o.ant_w0 * o.ant_w0));
    }
    return (float)(o.ant_J0 * G * T * cos(o.ant_omega * (t - o.ant_t0)));
}

__global__ void __launch_bounds__(256) k_antenna(const YeeArgs a)
{
    for (int box = 0; box < a.nboxes; ++box) {
        const BoxDev& b = a.boxes[box];
        const int j = b.oy.ant_j;
        if (j < 0)
            continue;
        const int64_t n = (int64_t)b.nx * b.nz;
        for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
             t += (int64_t)gridDim.x * blockDim.x) {
            const int x = (int)(t % b.nx), z = (int)(t / b.nx);
            b.J[padded_index(b, x, j, z)] += antenna_current(a, b, x, z);
        }
    }
}

// FOLD_Z false: the boxes are subdomain slabs, whose z guards went to their
// neighbours (and theirs came in as additions): no z images to fold.
template <int G, bool FOLD_Z>
__global__ void __launch_bounds__(256, 4) k_yee_e(const YeeArgs a)
{
    const BoxDev* bp;
    CellAt c = yee_cell(a, bp);
    if (!c.ok)
        return;
    const BoxDev& b = *bp;
    const int64_t pc = padded_cells(b);
    const int64_t sx = 1, sy = b.px, sz = (int64_t)b.px * b.py;
    const float* __restrict__ Bx = b.B;
    const float* __restrict__ By = b.B + pc;
    const float* __restrict__ Bz = b.B + 2 * pc;
    float* __restrict__ Ex = b.E;
    float* __restrict__ Ey = b.E + pc;
    float* __restrict__ Ez = b.E + 2 * pc;
    const float* __restrict__ J = b.J;
    const int z0 = c.z * kYeeZ;
    int ix[2], iy[2];
    const int nx = images(c.x, b.nx, G, GuardsOf<G>::hx, ix);
    const int ny = images(c.y, b.ny, G, GuardsOf<G>::hyz, iy);
    float jx[kYeeZ], jy[kYeeZ], jz[kYeeZ], cx[kYeeZ], cy[kYeeZ], cz[kYeeZ], ex[kYeeZ], ey[kYeeZ], ez[kYeeZ];
    float bxs[kYeeZ + 1], bys[kYeeZ + 1];
    {
        const int64_t i0 = pidx<G>(b, c.x, c.y, z0 - 1);
        bxs[0] = __ldg(Bx + i0);
        bys[0] = __ldg(By + i0);
    }
#pragma unroll
    for (int q = 0; q < kYeeZ; ++q) {
        const int64_t i = pidx<G>(b, c.x, c.y, z0 + q);
        int iz[2];
        const int nz = FOLD_Z ? images(z0 + q, b.nz, G, GuardsOf<G>::hyz, iz) : (iz[0] = z0 + q, 1);
        // fold the J guard images into the interior
        jx[q] = 0.f;
        jy[q] = 0.f;
        jz[q] = 0.f;
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int r = 0; r < 2; ++r)
                    if (k < nz && j < ny && r < nx) {
                        const int64_t g = pidx<G>(b, ix[r], iy[j], iz[k]);
                        jx[q] += J[g];
                        jy[q] += J[pc + g];
                        jz[q] += J[2 * pc + g];
                    }
        // Bx, By one plane down: the previous cell's own values (cells stacked in z)
        bxs[q + 1] = __ldg(Bx + i);
        bys[q + 1] = __ldg(By + i);
        const float bxv = bxs[q + 1], byv = bys[q + 1], bzv = __ldg(Bz + i);
        cx[q] = (bzv - __ldg(Bz + i - sy)) * a.ih[1] - (byv - bys[q]) * a.ih[2];
        cy[q] = (bxv - bxs[q]) * a.ih[2] - (bzv - __ldg(Bz + i - sx)) * a.ih[0];
        cz[q] = (byv - __ldg(By + i - sx)) * a.ih[0] - (bxv - __ldg(Bx + i - sy)) * a.ih[1];
        ex[q] = Ex[i];
        ey[q] = Ey[i];
        ez[q] = Ez[i];
    }
#pragma unroll
    for (int q = 0; q < kYeeZ; ++q) {
        // J is left as deposited (the step zeroes it before the push, and a
        // read of J folds the images the same way)
        c.z = z0 + q;
        store_images_g<G>(b, Ex, c, ex[q] + a.tau * (cx[q] - jx[q]));
        store_images_g<G>(b, Ey, c, ey[q] + a.tau * (cy[q] - jy[q]));
        store_images_g<G>(b, Ez, c, ez[q] + a.tau * (cz[q] - jz[q]));
    }
}

// ------------------------------------------------------------ fused field update
//
// The whole field half of the cycle in one kernel, from one buffer pair into
// the other: E^n, B^n and J are read from `src`, E^{n+1} and B^{n+1} (with
// their periodic guard images) are written into `dst`, so that no value is
// overwritten while a neighbouring cell still needs it.  Each block
// z-marches an output tile of kFusedTX x kFusedTY cells through a chunk of
// kFusedTZ planes.  Iteration s forms, with one block barrier after it,
//   B^{n+1/2}(s+1) on the tile and one cell around it (E^n planes s+1, s+2),
//   E^{n+1}(s)     on the tile and one cell above it in x and y
//                  (B^{n+1/2} planes s-1, s: earlier iterations),
//   B^{n+1}(s-2)   on the tile (E^{n+1} planes s-2, s-1: earlier iterations),
// so the three stages of an iteration depend only on earlier iterations and
// the intermediate B^{n+1/2} and E^{n+1} stay in shared memory; halo cells
// are formed again by the neighbouring tiles (and the first planes of a
// chunk by the chunk below).  The inputs of iteration s -- E^n(s+2), B^n(s+1)
// and J(s), each a plane tile of the three components -- arrive by tensor
// loads kFLook iterations ahead on one mbarrier; a thread waits for them and
// otherwise touches global memory only for its stores and for the few J
// guard images that fold into cells next to a box face.  HBM traffic per
// cell: E^n, B^n, J read and E^{n+1}, B^{n+1} written, 60 bytes (the three
// in-place kernels move 120); the halo rows come from L2.  The arithmetic of
// every value is that of k_yee_b, k_yee_e, k_yee_b.
constexpr int kFX = kFusedTX, kFY = kFusedTY, kFT = kFX * kFY;
constexpr int kFEX = kFusedEX, kFEY = kFY + 3;  // plane tile: cells x0-G .. x0-G+35, y0-1 .. y0+kFY+1
constexpr int kFSlot = ((3 * kFEY * kFEX + 31) / 32) * 32;  // floats, 128-byte slots
constexpr unsigned kFBytes = 3u * kFEY * kFEX * 4u;         // bytes of one plane tile
constexpr int kFLook = 3;                                    // bundles issued ahead
constexpr int kFRE = 8, kFRB = 4;  // E^n slots (>= kFLook + 3); B^n, J slots and mbarriers (>= kFLook + 1)
static_assert(kFRE >= kFLook + 3 && kFRB >= kFLook + 1 && !(kFRE & (kFRE - 1)) && !(kFRB & (kFRB - 1)),
              "power-of-two rings deep enough for the look-ahead");
constexpr int kHX = kFX + 2, kHY = kFY + 2, kHN = kHX * kHY;  // B^{n+1/2}: x0-1.., y0-1..
constexpr int kEX = kFX + 1, kEY = kFY + 1, kEN = kEX * kEY;  // E^{n+1}: x0.., y0..
constexpr int kHPer = (kHN + kFT - 1) / kFT, kEPer = (kEN + kFT - 1) / kFT;
static_assert(kFEX >= kFX + 4 && kFEX % 4 == 0, "plane rows reach x0 + kFX + 2 from a 16-byte start");

struct FusedSmem {
    float en[kFRE][kFSlot];  // E^n plane tiles [c][y][x]
    float bn[kFRB][kFSlot];  // B^n plane tiles
    float jn[kFRB][kFSlot];  // J plane tiles (as deposited; guard images folded by the reader)
    float bh[4][3][kHN];     // B^{n+1/2}, four planes [plane % 4][c][cell]
    float e1[4][3][kEN];     // E^{n+1}, four planes [plane % 4][c][cell]
    unsigned long long mb[kFRB];
    int abort;
};

struct FusedArgs {
    const BoxDev* src;
    const BoxDev* dst;
    const CUtensorMap* maps;  // [nboxes][3]: E, B, J plane maps over src
    const int* blk_off;
    int nboxes;
    float dt, tau;  // tau = dt / 2
    float ih[3];
    unsigned* status;
};

int fused_blocks(int nx, int ny, int nz)
{
    return ((nx + kFX - 1) / kFX) * ((ny + kFY - 1) / kFY) * ((nz + kFusedTZ - 1) / kFusedTZ);
}

template <int G>
__global__ void __launch_bounds__(kFT, 2) k_yee_fused(const FusedArgs a)
{
    extern __shared__ __align__(128) unsigned char fused_smem[];
    FusedSmem& sm = *reinterpret_cast<FusedSmem*>(fused_smem);
    const int box = find_box(a.blk_off, a.nboxes, blockIdx.x);
    // the box's geometry and arrays in registers (stores through the field
    // pointers could otherwise alias the table and force reloads)
    const BoxDev& bt = a.src[box];
    const int nx = bt.nx, ny = bt.ny, nz = bt.nz, px = bt.px, py = bt.py;
    const int64_t pc = (int64_t)px * py * bt.pz;
    const float* __restrict__ Jg = bt.J;
    float* __restrict__ Eo = a.dst[box].E;
    float* __restrict__ Bo = a.dst[box].B;
    constexpr int hx = GuardsOf<G>::hx, hyz = GuardsOf<G>::hyz;
    auto at = [&](int x, int y, int z) { return ((int64_t)(z + G) * py + (y + G)) * px + (x + G); };
    // the three components of interior cell (x, y, z) and of its guard images
    auto store3 = [&](float* F, int x, int y, int z, float v0, float v1, float v2) {
        int ix[2], iy[2], iz[2];
        const int cx = images(x, nx, G, hx, ix), cy = images(y, ny, G, hyz, iy), cz = images(z, nz, G, hyz, iz);
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int i = 0; i < 2; ++i)
                    if (k < cz && j < cy && i < cx) {
                        const int64_t g = at(ix[i], iy[j], iz[k]);
                        F[g] = v0;
                        F[pc + g] = v1;
                        F[2 * pc + g] = v2;
                    }
    };
    // interior cells away from every face have no images: one store each
    const int64_t plane = (int64_t)px * py;
    auto store3_fast = [&](float* F, bool col_plain, int64_t col, int x, int y, int z, float v0, float v1,
                           float v2) {
        if (col_plain && z >= hyz && z < nz - G) {
            const int64_t g = (int64_t)(z + G) * plane + col;
            F[g] = v0;
            F[pc + g] = v1;
            F[2 * pc + g] = v2;
        } else {
            store3(F, x, y, z, v0, v1, v2);
        }
    };
    const int local = blockIdx.x - a.blk_off[box];
    const int ntx = (nx + kFX - 1) / kFX, nty = (ny + kFY - 1) / kFY;
    const int x0 = (local % ntx) * kFX, y0 = ((local / ntx) % nty) * kFY;
    const int zc0 = (local / (ntx * nty)) * kFusedTZ, zc1 = min(zc0 + kFusedTZ, nz);
    const int tid = threadIdx.x;
    const CUtensorMap* maps = a.maps + 3 * box;
    // bundle k (k0 .. zc1 + 1): E^n(k+2) while k+2 <= zc1+1, B^n(k+1) while
    // zc0-1 <= k+1 <= zc1, J(k) while zc0 <= k <= zc1; E^n in slot
    // (k - k0) % kFRE, B^n and J in slot (k - k0) % kFRB, completing on that
    // slot's mbarrier as its ((k - k0) / kFRB)-th phase
    const int k0 = zc0 - 3, klast = zc1 + 1;
    int kiss = k0 - 1;  // tid 0: the last bundle issued
    auto issue = [&](int k) {
        kiss = k;
        const int e = (k - k0) & (kFRE - 1), r = (k - k0) & (kFRB - 1);
        const bool le = k + 2 <= zc1 + 1, lb = k + 1 >= zc0 - 1 && k + 1 <= zc1, lj = k >= zc0 && k <= zc1;
        unsigned long long* mb = &sm.mb[r];
        mbar_expect_tx(mb, kFBytes * ((le ? 1u : 0u) + (lb ? 1u : 0u) + (lj ? 1u : 0u)));
        if (le)
            tma_load_tile(sm.en[e], maps + 0, x0, y0 - 1 + G, k + 2 + G, mb);
        if (lb)
            tma_load_tile(sm.bn[r], maps + 1, x0, y0 - 1 + G, k + 1 + G, mb);
        if (lj)
            tma_load_tile(sm.jn[r], maps + 2, x0, y0 - 1 + G, k + G, mb);
    };
    if (tid == 0) {
        for (int r = 0; r < kFRB; ++r)
            mbar_init(&sm.mb[r], 1);
        fence_mbar_init();
        sm.abort = 0;
        for (int k = k0; k <= min(k0 + kFLook, klast); ++k)
            issue(k);
    }
    // J of the guard images of this thread's E^{n+1} cells other than the
    // position itself (zero away from the box faces), one plane ahead
    // (a column x, y inside [hx, nx - G) x [hyz, ny - G) and a plane inside
    // [hyz, nz - G) have no images: most cells skip at once)
    const auto inner = [](int v, int n, int h) { return v >= h && v < n - G; };
    bool col_plain[kEPer], col_in[kEPer];
#pragma unroll
    for (int k = 0; k < kEPer; ++k) {
        const int i = tid + k * kFT;
        col_plain[k] = inner(x0 + i % kEX, nx, hx) && inner(y0 + i / kEX, ny, hyz);
        col_in[k] = i < kEN && x0 + i % kEX <= nx && y0 + i / kEX <= ny;
    }
    auto fold_extra = [&](int s, float (&v)[kEPer][3]) {
        const bool plane_plain = inner(s, nz, hyz) || s < zc0 || s > zc1;
#pragma unroll
        for (int k = 0; k < kEPer; ++k) {
            v[k][0] = v[k][1] = v[k][2] = 0.0f;
            if ((col_plain[k] && plane_plain) || !col_in[k] || s < zc0 || s > zc1)
                continue;
            const int i = tid + k * kFT;
            const int x = x0 + i % kEX, y = y0 + i / kEX;
            int ix[2], iy[2], iz[2];
            const int cx = images(x < nx ? x : x - nx, nx, G, hx, ix);
            const int cy = images(y < ny ? y : y - ny, ny, G, hyz, iy);
            const int cz = images(s < nz ? s : s - nz, nz, G, hyz, iz);
            if (cx == 1 && cy == 1 && cz == 1)
                continue;
#pragma unroll
            for (int kk = 0; kk < 2; ++kk)
#pragma unroll
                for (int j = 0; j < 2; ++j)
#pragma unroll
                    for (int r = 0; r < 2; ++r)
                        if (kk < cz && j < cy && r < cx && !(ix[r] == x && iy[j] == y && iz[kk] == s)) {
                            const int64_t g = at(ix[r], iy[j], iz[kk]);
                            v[k][0] += __ldg(Jg + g);
                            v[k][1] += __ldg(Jg + pc + g);
                            v[k][2] += __ldg(Jg + 2 * pc + g);
                        }
        }
    };
    float jx[kEPer][3] = {}, jxn[kEPer][3] = {};
    __syncthreads();  // the mbarriers are initialised
    // bundle k0 (E^n(zc0-1) alone) before the loop, and a barrier after it:
    // its mbarrier is re-armed by the first iteration, for bundle k0 + kFRB
    bool timed_out = !mbar_wait(&sm.mb[0], 0u);
    __syncthreads();

    constexpr int EC = kFEY * kFEX;
    const float ih0 = a.ih[0], ih1 = a.ih[1], ih2 = a.ih[2], dt = a.dt, tau = a.tau;
    // this thread's cells, the same in every plane: stage 1 cells i1 (tile
    // index e1), stage 2 cells (tile index e2, B^{n+1/2} index h2, stored
    // when st2), stage 3 cell (E^{n+1} index e3, B^{n+1/2} index h3)
    int e1[kHPer], e2[kEPer], h2[kEPer];
    bool st2[kEPer];
    int64_t col2[kEPer];
    // (the stage 1 cells past the first kFT go to the last threads and the
    // stage 2 ones to the first, so that no warp takes both)
    int i1[kHPer];
#pragma unroll
    for (int k = 0; k < kHPer; ++k) {
        const int i = k == 0 ? tid : k * kFT + (kFT - 1 - tid);
        i1[k] = i;
        e1[k] = (i / kHX) * kFEX + i % kHX + G - 1;
    }
#pragma unroll
    for (int k = 0; k < kEPer; ++k) {
        const int i = tid + k * kFT, rx = i % kEX, ry = i / kEX;
        h2[k] = (ry + 1) * kHX + rx + 1;
        e2[k] = (ry + 1) * kFEX + rx + G;
        st2[k] = i < kEN && rx < kFX && ry < kFY && x0 + rx < nx && y0 + ry < ny;
        col2[k] = (int64_t)(y0 + ry + G) * px + (x0 + rx + G);
    }
    const int rx3 = tid % kFX, ry3 = tid / kFX;
    const int e3 = ry3 * kEX + rx3, h3 = (ry3 + 1) * kHX + rx3 + 1;
    const bool st3 = x0 + rx3 < nx && y0 + ry3 < ny;
    const bool plain3 = inner(x0 + rx3, nx, hx) && inner(y0 + ry3, ny, hyz);
    const int64_t col3 = (int64_t)(y0 + ry3 + G) * px + (x0 + rx3 + G);
    for (int s = zc0 - 2; s <= zc1 + 1; ++s) {
        if (tid == 0 && s + kFLook <= klast) {
            fence_proxy_async();  // the slots being refilled were read by generic loads
            issue(s + kFLook);
        }
        if (s >= zc0 - 1)
            fold_extra(s + 1, jxn);
        // the bundle of iteration s; its mbarrier was re-armed (at the top of
        // iteration s - kFRB + kFLook) only after every thread had waited on
        // that mbarrier's previous bundle and passed the barrier after it
        if (!mbar_wait(&sm.mb[(s - k0) & (kFRB - 1)], (unsigned)(((s - k0) / kFRB) & 1)))
            timed_out = true;
        if (timed_out)
            sm.abort = 1;
        // stage 1: B^{n+1/2}(s+1) = B^n - tau curl E^n
        if (s + 1 >= zc0 - 1 && s + 1 <= zc1) {
            const float* E1 = sm.en[(s - 1 - k0) & (kFRE - 1)];  // plane s+1 (bundle s-1)
            const float* E2 = sm.en[(s - k0) & (kFRE - 1)];      // plane s+2 (bundle s)
            const float* Bp = sm.bn[(s - k0) & (kFRB - 1)];      // B^n plane s+1
            float* H = sm.bh[(s + 1) & 3][0];
#pragma unroll
            for (int k = 0; k < kHPer; ++k) {
                const int i = i1[k];
                if (i < kHN) {
                    const int e = e1[k];  // cell (x, y) in the plane tiles
                    const float ex = E1[e], ey = E1[EC + e], ez = E1[2 * EC + e];
                    const float cx = (E1[2 * EC + e + kFEX] - ez) * ih1 - (E2[EC + e] - ey) * ih2;
                    const float cy = (E2[e] - ex) * ih2 - (E1[2 * EC + e + 1] - ez) * ih0;
                    const float cz = (E1[EC + e + 1] - ey) * ih0 - (E1[e + kFEX] - ex) * ih1;
                    H[i] = Bp[e] - tau * cx;
                    H[kHN + i] = Bp[EC + e] - tau * cy;
                    H[2 * kHN + i] = Bp[2 * EC + e] - tau * cz;
                }
            }
        }
        // stage 2: E^{n+1}(s) = E^n + dt (curl B^{n+1/2} - J)
        if (s >= zc0 && s <= zc1) {
            const float* H = sm.bh[s & 3][0];          // plane s
            const float* Hp = sm.bh[(s - 1) & 3][0];   // plane s - 1
            const float* E0 = sm.en[(s - 2 - k0) & (kFRE - 1)];  // E^n plane s (bundle s-2)
            const float* Jp = sm.jn[(s - k0) & (kFRB - 1)];      // J plane s
            float* X = sm.e1[s & 3][0];
#pragma unroll
            for (int k = 0; k < kEPer; ++k) {
                const int i = tid + k * kFT;
                if (i < kEN) {
                    const int h = h2[k], e = e2[k];
                    const float bxv = H[h], byv = H[kHN + h], bzv = H[2 * kHN + h];
                    const float cx = (bzv - H[2 * kHN + h - kHX]) * ih1 - (byv - Hp[kHN + h]) * ih2;
                    const float cy = (bxv - Hp[h]) * ih2 - (bzv - H[2 * kHN + h - 1]) * ih0;
                    const float cz = (byv - H[kHN + h - 1]) * ih0 - (bxv - H[h - kHX]) * ih1;
                    const float nex = E0[e] + dt * (cx - (Jp[e] + jx[k][0]));
                    const float ney = E0[EC + e] + dt * (cy - (Jp[EC + e] + jx[k][1]));
                    const float nez = E0[2 * EC + e] + dt * (cz - (Jp[2 * EC + e] + jx[k][2]));
                    X[i] = nex;
                    X[kEN + i] = ney;
                    X[2 * kEN + i] = nez;
                    if (st2[k] && s < zc1)
                        store3_fast(Eo, col_plain[k], col2[k], x0 + i % kEX, y0 + i / kEX, s, nex, ney, nez);
                }
            }
        }
        // stage 3: B^{n+1}(s-2) = B^{n+1/2} - tau curl E^{n+1}
        if (s - 2 >= zc0 && s - 2 < zc1) {
            if (st3) {
                const float* X0 = sm.e1[(s - 2) & 3][0];  // plane s - 2
                const float* X1 = sm.e1[(s - 1) & 3][0];  // plane s - 1
                const float* Hq = sm.bh[(s - 2) & 3][0];  // plane s - 2
                const int e = e3, h = h3;
                const float ex = X0[e], ey = X0[kEN + e], ez = X0[2 * kEN + e];
                const float cx = (X0[2 * kEN + e + kEX] - ez) * ih1 - (X1[kEN + e] - ey) * ih2;
                const float cy = (X1[e] - ex) * ih2 - (X0[2 * kEN + e + 1] - ez) * ih0;
                const float cz = (X0[kEN + e + 1] - ey) * ih0 - (X0[e + kEX] - ex) * ih1;
                store3_fast(Bo, plain3, col3, x0 + rx3, y0 + ry3, s - 2, Hq[h] - tau * cx, Hq[kHN + h] - tau * cy,
                            Hq[2 * kHN + h] - tau * cz);
            }
        }
        __syncthreads();
        if (sm.abort)
            break;
        if (s >= zc0 - 1)
#pragma unroll
            for (int k = 0; k < kEPer; ++k)
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    jx[k][c] = jxn[k][c];
    }
    if (sm.abort && tid == 0) {
        atomicOr(a.status, ST_TIMEOUT);
        // loads still in flight land before the block's shared memory goes
        // away: the last bundle issued on each mbarrier
        for (int k = max(k0, kiss - kFRB + 1); k <= kiss; ++k)
            mbar_wait(&sm.mb[(k - k0) & (kFRB - 1)], (unsigned)(((k - k0) / kFRB) & 1));
    }
}

size_t fused_smem_bytes() { return sizeof(FusedSmem); }

cudaError_t configure_yee_fused()
{
    cudaError_t e = cudaFuncSetAttribute(k_yee_fused<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(FusedSmem));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_yee_fused<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(FusedSmem));
    return e;
}

// y absorber: every E and B value whose staggered y position lies in a
// damping layer is multiplied by exp(-sigma d^2) (d = depth in the layer, 0
// at its inner edge, 1 at the face), images included.  Work: the 2A planes
// j < A and j >= ny - A of each box with a layer, 256 cells per block.
__device__ __forceinline__ float absorb_factor(float y, int ny, int A, float sigma)
{
    float depth = 0.0f;
    if (y < (float)A)
        depth = ((float)A - y) / (float)A;
    else if (y > (float)(ny - A))
        depth = (y - (float)(ny - A)) / (float)A;
    depth = fminf(depth, 1.0f);
    return expf(-sigma * depth * depth);
}

int absorber_blocks(const BoxDev& b)
{
    const int A = b.oy.abs_cells;
    if (A <= 0)
        return 0;
    const int64_t cells = (int64_t)2 * A * b.nx * b.nz;
    return (int)((cells + 255) / 256);
}

__global__ void __launch_bounds__(256) k_absorb_y(const BoxDev* boxes, const int* off, int nboxes)
{
    const int box = find_box(off, nboxes, blockIdx.x);
    const BoxDev& b = boxes[box];
    const int A = b.oy.abs_cells;
    const int64_t t = (int64_t)(blockIdx.x - off[box]) * 256 + threadIdx.x;
    if (A <= 0 || t >= (int64_t)2 * A * b.nx * b.nz)
        return;
    CellAt c;
    c.x = (int)(t % b.nx);
    const int p = (int)((t / b.nx) % (2 * A));
    c.z = (int)(t / ((int64_t)b.nx * 2 * A));
    c.y = p < A ? p : b.ny - 2 * A + p;
    c.ok = true;
    const int64_t pc = padded_cells(b);
    const int64_t i = padded_index(b, c.x, c.y, c.z);
    const float s = b.oy.abs_sigma;
    const float fi = absorb_factor((float)c.y, b.ny, A, s);          // Ex, Ez, By
    const float fh = absorb_factor((float)c.y + 0.5f, b.ny, A, s);   // Ey, Bx, Bz
    store_with_images(b, b.E, c, b.E[i] * fi);
    store_with_images(b, b.E + pc, c, b.E[pc + i] * fh);
    store_with_images(b, b.E + 2 * pc, c, b.E[2 * pc + i] * fi);
    store_with_images(b, b.B, c, b.B[i] * fh);
    store_with_images(b, b.B + pc, c, b.B[pc + i] * fi);
    store_with_images(b, b.B + 2 * pc, c, b.B[2 * pc + i] * fh);
}

cudaError_t launch_yee_mixed_part(const YeePlan& p, int part, cudaStream_t st)
{
    YeeArgs a{p.boxes, p.blk_off, p.nboxes, 0.5f * p.dt, {p.ih[0], p.ih[1], p.ih[2]},
              p.step_no, p.dt_d, {p.dx_d[0], p.dx_d[1], p.dx_d[2]}};
    dim3 blk(32, 8);
    auto yb = p.guard == 2 ? k_yee_b<2> : k_yee_b<1>;
    auto ye = p.guard == 2 ? (p.sub_z ? k_yee_e<2, false> : k_yee_e<2, true>)
                           : (p.sub_z ? k_yee_e<1, false> : k_yee_e<1, true>);
    if (part == 0) {
        yb<<<p.nblocks, blk, 0, st>>>(a);
    } else if (part == 1) {
        if (p.antenna)
            k_antenna<<<64, 256, 0, st>>>(a);
        a.tau = p.dt;
        ye<<<p.nblocks, blk, 0, st>>>(a);
    } else {
        yb<<<p.nblocks, blk, 0, st>>>(a);
        if (p.abs_nblocks > 0)
            k_absorb_y<<<p.abs_nblocks, 256, 0, st>>>(p.boxes, p.abs_off, p.nboxes);
    }
    return cudaGetLastError();
}

cudaError_t launch_yee_mixed_plan(const YeePlan& p, cudaStream_t st)
{
    for (int part = 0; part < 3; ++part) {
        const cudaError_t e = launch_yee_mixed_part(p, part, st);
        if (e != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

cudaError_t launch_yee_fused(const YeePlan& p, const FusedPlan& f, cudaStream_t st)
{
    if (p.antenna) {
        YeeArgs ya{f.src, p.blk_off, p.nboxes, p.dt, {p.ih[0], p.ih[1], p.ih[2]},
                   p.step_no, p.dt_d, {p.dx_d[0], p.dx_d[1], p.dx_d[2]}};
        k_antenna<<<64, 256, 0, st>>>(ya);
    }
    FusedArgs a{f.src, f.dst, f.maps, f.blk_off, p.nboxes, p.dt, 0.5f * p.dt, {p.ih[0], p.ih[1], p.ih[2]},
                f.status};
    if (p.guard == 2)
        k_yee_fused<2><<<f.nblocks, kFT, sizeof(FusedSmem), st>>>(a);
    else
        k_yee_fused<1><<<f.nblocks, kFT, sizeof(FusedSmem), st>>>(a);
    if (p.abs_nblocks > 0)
        k_absorb_y<<<p.abs_nblocks, 256, 0, st>>>(f.dst, p.abs_off, p.nboxes);
    return cudaGetLastError();
}

// ------------------------------------------------------------ subdomain halos

// Whole padded planes [p0, p0 + np) of the three components of F and a
// contiguous buffer [comp][plane][py][px]: mode 0 copies F to buf, 1 buf to
// F, 2 adds buf into F.  The planes of one component are contiguous in F
// too, so both sides are read and written in 16-byte pieces (px is a
// multiple of 4).
__global__ void k_halo_planes(const BoxDev b, float* F, int p0, int np, float* buf, int mode)
{
    const int64_t plane4 = (int64_t)b.px * b.py / 4;
    const int64_t per_comp = plane4 * np;
    const int64_t pc4 = padded_cells(b) / 4;
    float4* F4 = reinterpret_cast<float4*>(F);
    float4* B4 = reinterpret_cast<float4*>(buf);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < 3 * per_comp;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int comp = (int)(t / per_comp);
        const int64_t r = t - comp * per_comp;
        const int64_t f = comp * pc4 + (int64_t)p0 * plane4 + r;
        if (mode == 0) {
            B4[t] = F4[f];
        } else if (mode == 1) {
            F4[f] = B4[t];
        } else {
            const float4 v = B4[t];
            float4 u = F4[f];
            u.x += v.x;
            u.y += v.y;
            u.z += v.z;
            u.w += v.w;
            F4[f] = u;
        }
    }
}

cudaError_t launch_halo_planes(const BoxDev& b, float* F, int p0, int np, float* buf, int mode,
                               cudaStream_t st)
{
    if (np <= 0)
        return cudaSuccess;
    const int64_t n4 = 3 * (int64_t)b.px * b.py / 4 * np;
    const int blocks = (int)std::min<int64_t>((n4 + 255) / 256, 2048);
    k_halo_planes<<<blocks, 256, 0, st>>>(b, F, p0, np, buf, mode);
    return cudaGetLastError();
}

// Moving window: F (3 components) takes the values of scratch (a copy of F)
// `cells` planes higher; the planes entering at the top are zero; images
// rewritten.
__global__ void k_shift_fields(const BoxDev b, float* F, const float* scratch, int cells)
{
    const int64_t n = (int64_t)b.nx * b.ny * b.nz;
    const int64_t pc = padded_cells(b);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < 3 * n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int comp = (int)(t / n);
        const int64_t r = t - comp * n;
        CellAt c;
        c.x = (int)(r % b.nx);
        c.y = (int)((r / b.nx) % b.ny);
        c.z = (int)(r / ((int64_t)b.nx * b.ny));
        c.ok = true;
        const float v = c.y + cells < b.ny ? scratch[comp * pc + padded_index(b, c.x, c.y + cells, c.z)] : 0.0f;
        store_with_images(b, F + comp * pc, c, v);
    }
}

cudaError_t launch_shift_fields(const BoxDev& b, float* F, const float* scratch, int cells,
                                cudaStream_t st)
{
    k_shift_fields<<<1024, 256, 0, st>>>(b, F, scratch, cells);
    return cudaGetLastError();
}

// ------------------------------------------------------------ import/export

// src: FP64 [3][nz][ny][nx] on the device -> padded FP32 field with images.
__global__ void k_fields_to_padded(const BoxDev b, float* F, const double* src)
{
    const int64_t n = (int64_t)b.nx * b.ny * b.nz;
    const int64_t pc = padded_cells(b);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < 3 * n;
         t += (int64_t)gridDim.x * blockDim.x) {
        int comp = (int)(t / n);
        int64_t r = t - comp * n;
        CellAt c;
        c.x = (int)(r % b.nx);
        c.y = (int)((r / b.nx) % b.ny);
        c.z = (int)(r / ((int64_t)b.nx * b.ny));
        store_with_images(b, F + comp * pc, c, (float)src[t]);
    }
}

// fold: sum the periodic images (the current, whose guards hold deposits
// that crossed the seam), in the order of the E update's fold.
__global__ void k_fields_from_padded(const BoxDev b, const float* F, double* dst, int fold)
{
    const int64_t n = (int64_t)b.nx * b.ny * b.nz;
    const int64_t pc = padded_cells(b);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < 3 * n;
         t += (int64_t)gridDim.x * blockDim.x) {
        int comp = (int)(t / n);
        int64_t r = t - comp * n;
        int x = (int)(r % b.nx), y = (int)((r / b.nx) % b.ny), z = (int)(r / ((int64_t)b.nx * b.ny));
        const float* Fc = F + comp * pc;
        if (!fold) {
            dst[t] = (double)Fc[padded_index(b, x, y, z)];
            continue;
        }
        int ix[2], iy[2], iz[2];
        const int nx = images_x(b, x, ix), ny = images_y(b, y, iy);
        const int nz = b.sub_z ? (iz[0] = z, 1) : images_z(b, z, iz);
        float v = 0.0f;
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int q = 0; q < nx; ++q)
                    v += Fc[padded_index(b, ix[q], iy[j], iz[k])];
        dst[t] = (double)v;
    }
}

cudaError_t launch_fields_to_padded(const BoxDev& b, int which, const double* src, cudaStream_t st)
{
    float* F = which == 0 ? b.E : (which == 1 ? b.B : b.J);
    k_fields_to_padded<<<1024, 256, 0, st>>>(b, F, src);
    return cudaGetLastError();
}

cudaError_t launch_fields_from_padded(const BoxDev& b, int which, double* dst, cudaStream_t st)
{
    const float* F = which == 0 ? b.E : (which == 1 ? b.B : b.J);
    k_fields_from_padded<<<1024, 256, 0, st>>>(b, F, dst, which == 2);
    return cudaGetLastError();
}

// ------------------------------------------------------------ FP64 diagnostics

__device__ __forceinline__ double block_sum(double v)
{
    __shared__ double s[32];
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0)
        s[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x + 31) / 32; ++i)
            r += s[i];
    __syncthreads();
    return r;
}

__global__ void k_diag_fields(const BoxDev b, double* out, double vol)
{
    const int64_t n = (int64_t)b.nx * b.ny * b.nz;
    const int64_t pc = padded_cells(b);
    double acc = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        int x = (int)(t % b.nx), y = (int)((t / b.nx) % b.ny), z = (int)(t / ((int64_t)b.nx * b.ny));
        int64_t i = padded_index(b, x, y, z);
        for (int c = 0; c < 3; ++c) {
            double e = b.E[c * pc + i], m = b.B[c * pc + i];
            acc += e * e + m * m;
        }
    }
    double s = block_sum(acc);
    if (threadIdx.x == 0)
        atomicAdd(out, 0.5 * s * vol);
}

// Shape weights in FP64 for the charge density (same shapes as the push).
__device__ __forceinline__ double shape64(int shape, double d)
{
    double a = fabs(d);
    if (shape == 1)
        return a < 1.0 ? 1.0 - a : 0.0;
    if (shape == 3) {  // PCS
        if (a < 1.0)
            return (4.0 - 6.0 * a * a + 3.0 * a * a * a) / 6.0;
        return a < 2.0 ? (2.0 - a) * (2.0 - a) * (2.0 - a) / 6.0 : 0.0;
    }
    if (a <= 0.5)
        return 0.75 - a * a;
    return a < 1.5 ? 0.5 * (1.5 - a) * (1.5 - a) : 0.0;
}

// One CTA per supercell of the box: kinetic energy, charge, and the charge
// density deposited (FP64 atomics) into rho[nz][ny][nx].
__global__ void k_diag_particles(const StepDev d, int box, double* rho, double* out, double ivol)
{
    const BoxDev b = d.boxes[box];
    const int loc = blockIdx.x;
    const int g = b.sc_base + loc;
    const int scx = loc % b.nscx, scy = (loc / b.nscx) % b.nscy, scz = loc / (b.nscx * b.nscy);
    double ekin = 0.0, q = 0.0;
    for (int s = 0; s < d.nspecies; ++s) {
        const SpeciesDev sp = d.sp[s];
        const int L = s * d.nsc + g;
        const int n = d.count[L];
        const int* ft = d.ftab + d.foff[L];
        const double mass = (double)sp.m;
        for (int p = threadIdx.x; p < n; p += blockDim.x) {
            const int64_t idx = (int64_t)ft[p >> d.log2S] * d.S + (p & (d.S - 1));
            const double ux = d.ux[idx], uy = d.uy[idx], uz = d.uz[idx], w = d.w[idx];
            const double u2 = ux * ux + uy * uy + uz * uz;
            ekin += w * mass * (u2 / (sqrt(1.0 + u2) + 1.0));
            q += (double)sp.q * w;
            const int cell = d.cell[idx];
            const double pos[3] = {(double)(scx * d.LX + cell % d.LX) + (double)d.ox[idx],
                                   (double)(scy * d.LY + (cell / d.LX) % d.LY) + (double)d.oy[idx],
                                   (double)(scz * d.LZ + cell / (d.LX * d.LY)) + (double)d.oz[idx]};
            int base[3];
            double wt[3][4];
            const int Nd[3] = {b.nx, b.ny, b.nz};
            for (int a = 0; a < 3; ++a) {
                base[a] = (int)floor(pos[a]) - 1;
                for (int k = 0; k < 4; ++k)
                    wt[a][k] = shape64(sp.shape, pos[a] - (double)(base[a] + k));
            }
            const double qw = (double)sp.q * w * ivol;
            for (int kz = 0; kz < 4; ++kz)
                for (int ky = 0; ky < 4; ++ky)
                    for (int kx = 0; kx < 4; ++kx) {
                        double v = wt[0][kx] * wt[1][ky] * wt[2][kz];
                        if (v == 0.0)
                            continue;
                        int X = (base[0] + kx + Nd[0]) % Nd[0];
                        int Y = (base[1] + ky + Nd[1]) % Nd[1];
                        int Z = (base[2] + kz + Nd[2]) % Nd[2];
                        atomicAdd(rho + ((int64_t)Z * b.ny + Y) * b.nx + X, qw * v);
                    }
        }
    }
    double se = block_sum(ekin);
    double sq = block_sum(q);
    if (threadIdx.x == 0) {
        atomicAdd(out + 1, se);
        atomicAdd(out + 2, sq);
    }
}

__global__ void k_diag_gauss(const BoxDev b, const double* rho, double rho_bg, double ih0, double ih1,
                             double ih2, unsigned long long* maxbits)
{
    const int64_t n = (int64_t)b.nx * b.ny * b.nz;
    const int64_t pc = padded_cells(b);
    double m = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        int x = (int)(t % b.nx), y = (int)((t / b.nx) % b.ny), z = (int)(t / ((int64_t)b.nx * b.ny));
        // a subdomain slab's charge density near its z faces misses the
        // neighbour's particles: its residual is taken 3 planes inside
        if (b.sub_z && (z < 3 || z >= b.nz - 3))
            continue;
        int64_t i = padded_index(b, x, y, z);
        double div = ((double)b.E[i] - (double)b.E[i - 1]) * ih0 +
                     ((double)b.E[pc + i] - (double)b.E[pc + i - b.px]) * ih1 +
                     ((double)b.E[2 * pc + i] - (double)b.E[2 * pc + i - (int64_t)b.px * b.py]) * ih2;
        m = fmax(m, fabs(div - rho[t] - rho_bg));
    }
    for (int o = 16; o > 0; o >>= 1)
        m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0)
        atomicMax(maxbits, (unsigned long long)__double_as_longlong(m));
}

cudaError_t launch_diag_mixed(const StepDev& d, const BoxDev& hb, int box, double rho_bg,
                              double* rho_scratch, double* out, const double h[3], cudaStream_t st)
{
    const int64_t n = (int64_t)hb.nx * hb.ny * hb.nz;
    cudaError_t e = cudaMemsetAsync(rho_scratch, 0, sizeof(double) * n, st);
    if (e != cudaSuccess)
        return e;
    e = cudaMemsetAsync(out, 0, sizeof(double) * 4, st);
    if (e != cudaSuccess)
        return e;
    const double vol = h[0] * h[1] * h[2];
    k_diag_fields<<<512, 256, 0, st>>>(hb, out, vol);
    k_diag_particles<<<hb.nscx * hb.nscy * hb.nscz, 128, 0, st>>>(d, box, rho_scratch, out, 1.0 / vol);
    k_diag_gauss<<<512, 256, 0, st>>>(hb, rho_scratch, rho_bg, 1.0 / h[0], 1.0 / h[1], 1.0 / h[2],
                                      reinterpret_cast<unsigned long long*>(out + 3));
    return cudaGetLastError();
}

}  // namespace pic
