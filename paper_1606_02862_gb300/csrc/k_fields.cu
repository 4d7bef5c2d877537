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
