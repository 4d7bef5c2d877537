// k_plain.cu -- the plain FP64 form of the PIC step: absolute FP64 particle
// positions in unsorted SoA arrays, FP64 fields without guards (periodic
// indices wrap), one thread per particle, current deposited straight into
// global memory with FP64 atomics, one box per launch.  It computes the same
// cycle as the mixed form (Sec. 4: gather with the particle shape, Boris,
// Esirkepov, Yee) and serves as the straightforward GPU baseline the mixed,
// supercell-sorted form is measured against.
#include "pic_internal.cuh"
#include "plain.cuh"

#include <cmath>

namespace pic {

__device__ __forceinline__ int wrapi(int i, int n)
{
    i %= n;
    return i < 0 ? i + n : i;
}

__device__ __forceinline__ double S64(int shape, double d)
{
    double a = fabs(d);
    if (shape == 1)
        return a < 1.0 ? 1.0 - a : 0.0;
    if (a <= 0.5)
        return 0.75 - a * a;
    return a < 1.5 ? 0.5 * (1.5 - a) * (1.5 - a) : 0.0;
}

// Weights of a component sampled at node + s (s = 0 or 1/2) along one axis:
// first node and NW weights.  red: one order lower (the energy-conserving
// gather along a staggered axis), placed in the same window: CIC inside the
// TSC window, nearest grid point inside the CIC window.
template <int SHAPE>
__device__ __forceinline__ int axis_weights(double x, double s, double* wt, bool red)
{
    if (SHAPE == 2) {
        double xs = x - s;
        double n0 = floor(xs + 0.5);
        double dd = xs - n0;
        if (red) {  // CIC between floor(xs) and floor(xs) + 1
            const bool below = dd < 0.0;  // floor(xs) = n0 - 1
            const double f = below ? dd + 1.0 : dd;
            wt[0] = below ? 1.0 - f : 0.0;
            wt[1] = below ? f : 1.0 - f;
            wt[2] = below ? 0.0 : f;
        } else {
            double a = 0.5 - dd, c = 0.5 + dd;
            wt[0] = 0.5 * a * a;
            wt[1] = 0.75 - dd * dd;
            wt[2] = 0.5 * c * c;
        }
        return (int)n0 - 1;
    } else {
        double xs = x - s;
        double n0 = floor(xs);
        double f = xs - n0;
        if (red) {  // nearest of n0, n0 + 1 (a tie goes up)
            wt[0] = f < 0.5 ? 1.0 : 0.0;
            wt[1] = f < 0.5 ? 0.0 : 1.0;
        } else {
            wt[0] = 1.0 - f;
            wt[1] = f;
        }
        return (int)n0;
    }
}

template <int SHAPE>
__device__ __forceinline__ double gather64(const double* __restrict__ F, int nx, int ny, int nz,
                                           double x, double y, double z, double sx, double sy,
                                           double sz, bool ec)
{
    constexpr int NW = SHAPE == 2 ? 3 : 2;
    double wx[NW], wy[NW], wz[NW];
    int bx = axis_weights<SHAPE>(x, sx, wx, ec && sx != 0.0);
    int by = axis_weights<SHAPE>(y, sy, wy, ec && sy != 0.0);
    int bz = axis_weights<SHAPE>(z, sz, wz, ec && sz != 0.0);
    double acc = 0.0;
#pragma unroll
    for (int c = 0; c < NW; ++c) {
        int Z = wrapi(bz + c, nz);
#pragma unroll
        for (int b = 0; b < NW; ++b) {
            int Y = wrapi(by + b, ny);
            const double* row = F + ((int64_t)Z * ny + Y) * nx;
            double r = 0.0;
#pragma unroll
            for (int a = 0; a < NW; ++a)
                r += __ldg(row + wrapi(bx + a, nx)) * wx[a];
            acc += r * wy[b] * wz[c];
        }
    }
    return acc;
}

template <int SHAPE>
__global__ void __launch_bounds__(256) k_plain_push(const PlainPushArgs a)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.n)
        return;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int64_t nc = (int64_t)nx * ny * nz;
    const double x0 = a.x[i], y0 = a.y[i], z0 = a.z[i];
    const bool ec = a.ec != 0;
    const double Ex = gather64<SHAPE>(a.E, nx, ny, nz, x0, y0, z0, 0.5, 0.0, 0.0, ec);
    const double Ey = gather64<SHAPE>(a.E + nc, nx, ny, nz, x0, y0, z0, 0.0, 0.5, 0.0, ec);
    const double Ez = gather64<SHAPE>(a.E + 2 * nc, nx, ny, nz, x0, y0, z0, 0.0, 0.0, 0.5, ec);
    const double Bx = gather64<SHAPE>(a.B, nx, ny, nz, x0, y0, z0, 0.0, 0.5, 0.5, ec);
    const double By = gather64<SHAPE>(a.B + nc, nx, ny, nz, x0, y0, z0, 0.5, 0.0, 0.5, ec);
    const double Bz = gather64<SHAPE>(a.B + 2 * nc, nx, ny, nz, x0, y0, z0, 0.5, 0.5, 0.0, ec);

    // relativistic Boris push
    const double eps = a.eps;
    double ux = a.ux[i], uy = a.uy[i], uz = a.uz[i];
    double umx = ux + eps * Ex, umy = uy + eps * Ey, umz = uz + eps * Ez;
    double gm = sqrt(1.0 + umx * umx + umy * umy + umz * umz);
    double tx = eps * Bx / gm, ty = eps * By / gm, tz = eps * Bz / gm;
    double f = 2.0 / (1.0 + tx * tx + ty * ty + tz * tz);
    double sx = f * tx, sy = f * ty, sz = f * tz;
    double upx = umx + (umy * tz - umz * ty);
    double upy = umy + (umz * tx - umx * tz);
    double upz = umz + (umx * ty - umy * tx);
    ux = umx + (upy * sz - upz * sy) + eps * Ex;
    uy = umy + (upz * sx - upx * sz) + eps * Ey;
    uz = umz + (upx * sy - upy * sx) + eps * Ez;
    double g = sqrt(1.0 + ux * ux + uy * uy + uz * uz);
    double D[3] = {a.move[0] * ux / g, a.move[1] * uy / g, a.move[2] * uz / g};
    if (!(fabs(D[0]) < 0.5 && fabs(D[1]) < 0.5 && fabs(D[2]) < 0.5)) {
        atomicOr(a.status, ST_PARTICLE);
        D[0] = D[1] = D[2] = 0.0;
        ux = uy = uz = 0.0;
    }
    const double p0[3] = {x0, y0, z0};
    // Esirkepov on the window of 4 integer nodes floor(x0)-1 .. floor(x0)+2
    int base[3];
    double S0[3][4], DS[3][4];
    for (int d = 0; d < 3; ++d) {
        double c0 = floor(p0[d]);
        base[d] = (int)c0 - 1;
        for (int k = 0; k < 4; ++k) {
            double node = c0 - 1.0 + k;
            S0[d][k] = S64(SHAPE, p0[d] - node);
            DS[d][k] = S64(SHAPE, p0[d] + D[d] - node) - S0[d][k];
        }
    }
    const double w = a.w[i];
    const int Nd[3] = {nx, ny, nz};
    for (int d = 0; d < 3; ++d) {
        const int e = (d + 1) % 3, h = (d + 2) % 3;
        const double coef = a.jcoef[d] * w;
        double* Jd = a.J + d * nc;
        double P[3];
        P[0] = DS[d][0];
        P[1] = P[0] + DS[d][1];
        P[2] = P[1] + DS[d][2];
        for (int kh = 0; kh < 4; ++kh)
            for (int ke = 0; ke < 4; ++ke) {
                double T = S0[e][ke] * S0[h][kh] + 0.5 * (DS[e][ke] * S0[h][kh] + S0[e][ke] * DS[h][kh]) +
                           DS[e][ke] * DS[h][kh] / 3.0;
                T *= coef;
                if (T == 0.0)
                    continue;
                for (int kd = 0; kd < 3; ++kd) {
                    if (P[kd] == 0.0)
                        continue;
                    int idx[3];
                    idx[d] = wrapi(base[d] + kd, Nd[d]);
                    idx[e] = wrapi(base[e] + ke, Nd[e]);
                    idx[h] = wrapi(base[h] + kh, Nd[h]);
                    atomicAdd(Jd + ((int64_t)idx[2] * ny + idx[1]) * nx + idx[0], P[kd] * T);
                }
            }
    }
    double out[3];
    for (int d = 0; d < 3; ++d) {
        double v = p0[d] + D[d];
        double N = (double)Nd[d];
        if (v >= N)
            v -= N;
        else if (v < 0.0)
            v += N;
        if (v >= N)
            v = 0.0;
        out[d] = v;
    }
    a.x[i] = out[0];
    a.y[i] = out[1];
    a.z[i] = out[2];
    a.ux[i] = ux;
    a.uy[i] = uy;
    a.uz[i] = uz;
}

cudaError_t launch_plain_push(const PlainPushArgs& a, int shape, cudaStream_t st)
{
    if (a.n == 0)
        return cudaSuccess;
    int blocks = (int)((a.n + 255) / 256);
    if (shape == 2)
        k_plain_push<2><<<blocks, 256, 0, st>>>(a);
    else
        k_plain_push<1><<<blocks, 256, 0, st>>>(a);
    return cudaGetLastError();
}

// ------------------------------------------------------------ Yee, FP64

__global__ void k_plain_yee_b(PlainYeeArgs a, double tau)
{
    const int64_t nc = (int64_t)a.nx * a.ny * a.nz;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nc;
         t += (int64_t)gridDim.x * blockDim.x) {
        int x = (int)(t % a.nx), y = (int)((t / a.nx) % a.ny), z = (int)(t / ((int64_t)a.nx * a.ny));
        int64_t xp = t - x + wrapi(x + 1, a.nx);
        int64_t yp = t + ((int64_t)wrapi(y + 1, a.ny) - y) * a.nx;
        int64_t zp = t + ((int64_t)wrapi(z + 1, a.nz) - z) * a.nx * a.ny;
        const double *Ex = a.E, *Ey = a.E + nc, *Ez = a.E + 2 * nc;
        double cx = (Ez[yp] - Ez[t]) * a.ih[1] - (Ey[zp] - Ey[t]) * a.ih[2];
        double cy = (Ex[zp] - Ex[t]) * a.ih[2] - (Ez[xp] - Ez[t]) * a.ih[0];
        double cz = (Ey[xp] - Ey[t]) * a.ih[0] - (Ex[yp] - Ex[t]) * a.ih[1];
        a.B[t] -= tau * cx;
        a.B[nc + t] -= tau * cy;
        a.B[2 * nc + t] -= tau * cz;
    }
}

__global__ void k_plain_yee_e(PlainYeeArgs a, double dt)
{
    const int64_t nc = (int64_t)a.nx * a.ny * a.nz;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nc;
         t += (int64_t)gridDim.x * blockDim.x) {
        int x = (int)(t % a.nx), y = (int)((t / a.nx) % a.ny), z = (int)(t / ((int64_t)a.nx * a.ny));
        int64_t xm = t - x + wrapi(x - 1, a.nx);
        int64_t ym = t + ((int64_t)wrapi(y - 1, a.ny) - y) * a.nx;
        int64_t zm = t + ((int64_t)wrapi(z - 1, a.nz) - z) * a.nx * a.ny;
        const double *Bx = a.B, *By = a.B + nc, *Bz = a.B + 2 * nc;
        double cx = (Bz[t] - Bz[ym]) * a.ih[1] - (By[t] - By[zm]) * a.ih[2];
        double cy = (Bx[t] - Bx[zm]) * a.ih[2] - (Bz[t] - Bz[xm]) * a.ih[0];
        double cz = (By[t] - By[xm]) * a.ih[0] - (Bx[t] - Bx[ym]) * a.ih[1];
        a.E[t] += dt * (cx - a.J[t]);
        a.E[nc + t] += dt * (cy - a.J[nc + t]);
        a.E[2 * nc + t] += dt * (cz - a.J[2 * nc + t]);
    }
}

cudaError_t launch_plain_yee(const PlainYeeArgs& a, double dt, cudaStream_t st)
{
    k_plain_yee_b<<<2048, 256, 0, st>>>(a, 0.5 * dt);
    k_plain_yee_e<<<2048, 256, 0, st>>>(a, dt);
    k_plain_yee_b<<<2048, 256, 0, st>>>(a, 0.5 * dt);
    return cudaGetLastError();
}

// ------------------------------------------------------------ load / diagnostics

__global__ void k_plain_load(int64_t n, const double* x, const double* u, const double* w,
                             int nx, int ny, int nz, double* X, double* Y, double* Z, double* UX,
                             double* UY, double* UZ, double* W, int* pid, int id_base,
                             unsigned* status)
{
    const int Nd[3] = {nx, ny, nz};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double p[3];
        bool bad = false;
        for (int d = 0; d < 3; ++d) {
            double v = x[3 * i + d];
            if (!isfinite(v) || !isfinite(u[3 * i + d]))
                bad = true;
            double N = (double)Nd[d];
            v = v - N * floor(v / N);
            if (!(v < N) || !(v >= 0.0))
                v = 0.0;
            p[d] = v;
        }
        double wv = w ? w[i] : 1.0;
        if (!isfinite(wv))
            bad = true;
        if (bad)
            atomicOr(status, ST_PARTICLE);
        X[i] = p[0];
        Y[i] = p[1];
        Z[i] = p[2];
        UX[i] = u[3 * i];
        UY[i] = u[3 * i + 1];
        UZ[i] = u[3 * i + 2];
        W[i] = wv;
        if (pid)
            pid[i] = id_base + (int)i;
    }
}

cudaError_t launch_plain_load(int64_t n, const double* x, const double* u, const double* w, int nx,
                              int ny, int nz, double* X, double* Y, double* Z, double* UX,
                              double* UY, double* UZ, double* W, int* pid, int id_base,
                              unsigned* status, cudaStream_t st)
{
    if (n == 0)
        return cudaSuccess;
    int blocks = (int)std::min<int64_t>((n + 255) / 256, 8192);
    k_plain_load<<<blocks, 256, 0, st>>>(n, x, u, w, nx, ny, nz, X, Y, Z, UX, UY, UZ, W, pid,
                                         id_base, status);
    return cudaGetLastError();
}

// interleave SoA FP64 particles into n x 3 host layout on the device
__global__ void k_plain_interleave(int64_t n, const double* X, const double* Y, const double* Z,
                                   double* out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        out[3 * i] = X[i];
        out[3 * i + 1] = Y[i];
        out[3 * i + 2] = Z[i];
    }
}

cudaError_t launch_plain_interleave(int64_t n, const double* X, const double* Y, const double* Z,
                                    double* out, cudaStream_t st)
{
    if (n == 0)
        return cudaSuccess;
    int blocks = (int)std::min<int64_t>((n + 255) / 256, 8192);
    k_plain_interleave<<<blocks, 256, 0, st>>>(n, X, Y, Z, out);
    return cudaGetLastError();
}

__device__ __forceinline__ double block_sum64(double v)
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

__global__ void k_plain_diag_fields(int64_t nc, const double* E, const double* B, double* out,
                                    double vol)
{
    double acc = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < 3 * nc;
         t += (int64_t)gridDim.x * blockDim.x)
        acc += E[t] * E[t] + B[t] * B[t];
    double s = block_sum64(acc);
    if (threadIdx.x == 0)
        atomicAdd(out, 0.5 * s * vol);
}

__global__ void k_plain_diag_particles(PlainPushArgs a, int shape, double mass, double q,
                                       double ivol, double* rho, double* out)
{
    double ek = 0.0, qs = 0.0;
    const int Nd[3] = {a.nx, a.ny, a.nz};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double ux = a.ux[i], uy = a.uy[i], uz = a.uz[i], w = a.w[i];
        double u2 = ux * ux + uy * uy + uz * uz;
        ek += w * mass * (u2 / (sqrt(1.0 + u2) + 1.0));
        qs += q * w;
        const double pos[3] = {a.x[i], a.y[i], a.z[i]};
        int base[3];
        double wt[3][4];
        for (int d = 0; d < 3; ++d) {
            base[d] = (int)floor(pos[d]) - 1;
            for (int k = 0; k < 4; ++k)
                wt[d][k] = S64(shape, pos[d] - (double)(base[d] + k));
        }
        for (int kz = 0; kz < 4; ++kz)
            for (int ky = 0; ky < 4; ++ky)
                for (int kx = 0; kx < 4; ++kx) {
                    double v = wt[0][kx] * wt[1][ky] * wt[2][kz];
                    if (v == 0.0)
                        continue;
                    int X = wrapi(base[0] + kx, Nd[0]), Y = wrapi(base[1] + ky, Nd[1]),
                        Z = wrapi(base[2] + kz, Nd[2]);
                    atomicAdd(rho + ((int64_t)Z * a.ny + Y) * a.nx + X, q * w * ivol * v);
                }
    }
    double s1 = block_sum64(ek);
    double s2 = block_sum64(qs);
    if (threadIdx.x == 0) {
        atomicAdd(out + 1, s1);
        atomicAdd(out + 2, s2);
    }
}

__global__ void k_plain_diag_gauss(PlainYeeArgs a, const double* rho, double rho_bg,
                                   unsigned long long* maxbits)
{
    const int64_t nc = (int64_t)a.nx * a.ny * a.nz;
    double m = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nc;
         t += (int64_t)gridDim.x * blockDim.x) {
        int x = (int)(t % a.nx), y = (int)((t / a.nx) % a.ny), z = (int)(t / ((int64_t)a.nx * a.ny));
        int64_t xm = t - x + wrapi(x - 1, a.nx);
        int64_t ym = t + ((int64_t)wrapi(y - 1, a.ny) - y) * a.nx;
        int64_t zm = t + ((int64_t)wrapi(z - 1, a.nz) - z) * a.nx * a.ny;
        double div = (a.E[t] - a.E[xm]) * a.ih[0] + (a.E[nc + t] - a.E[nc + ym]) * a.ih[1] +
                     (a.E[2 * nc + t] - a.E[2 * nc + zm]) * a.ih[2];
        m = fmax(m, fabs(div - rho[t] - rho_bg));
    }
    for (int o = 16; o > 0; o >>= 1)
        m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0)
        atomicMax(maxbits, (unsigned long long)__double_as_longlong(m));
}

cudaError_t launch_plain_diag_fields(const PlainYeeArgs& a, double* out, double vol, cudaStream_t st)
{
    int64_t nc = (int64_t)a.nx * a.ny * a.nz;
    k_plain_diag_fields<<<512, 256, 0, st>>>(nc, a.E, a.B, out, vol);
    return cudaGetLastError();
}

cudaError_t launch_plain_diag_particles(const PlainPushArgs& a, int shape, double mass, double q,
                                        double ivol, double* rho, double* out, cudaStream_t st)
{
    if (a.n == 0)
        return cudaSuccess;
    k_plain_diag_particles<<<512, 256, 0, st>>>(a, shape, mass, q, ivol, rho, out);
    return cudaGetLastError();
}

cudaError_t launch_plain_diag_gauss(const PlainYeeArgs& a, const double* rho, double rho_bg,
                                    double* out, cudaStream_t st)
{
    k_plain_diag_gauss<<<512, 256, 0, st>>>(a, rho, rho_bg,
                                            reinterpret_cast<unsigned long long*>(out + 3));
    return cudaGetLastError();
}

}  // namespace pic
