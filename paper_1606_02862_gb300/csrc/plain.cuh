// plain.cuh -- argument blocks of the plain FP64 kernels (k_plain.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pic {

struct PlainPushArgs {
    int nx, ny, nz;
    int64_t n;
    const double* E;  // [3][nz][ny][nx]
    const double* B;
    double* J;
    double *x, *y, *z, *ux, *uy, *uz, *w;  // SoA particles
    double eps;       // q dt / (2 m)
    double jcoef[3];  // -q h_d / (V dt)
    double move[3];   // dt / h_d
    unsigned* status;
    int ec;           // energy-conserving gather
};

struct PlainYeeArgs {
    int nx, ny, nz;
    double* E;
    double* B;
    const double* J;
    double ih[3];
};

cudaError_t launch_plain_push(const PlainPushArgs& a, int shape, cudaStream_t st);
cudaError_t launch_plain_yee(const PlainYeeArgs& a, double dt, cudaStream_t st);
cudaError_t launch_plain_load(int64_t n, const double* x, const double* u, const double* w, int nx,
                              int ny, int nz, double* X, double* Y, double* Z, double* UX,
                              double* UY, double* UZ, double* W, int* pid, int id_base,
                              unsigned* status, cudaStream_t st);
cudaError_t launch_plain_interleave(int64_t n, const double* X, const double* Y, const double* Z,
                                    double* out, cudaStream_t st);
cudaError_t launch_plain_diag_fields(const PlainYeeArgs& a, double* out, double vol, cudaStream_t st);
cudaError_t launch_plain_diag_particles(const PlainPushArgs& a, int shape, double mass, double q,
                                        double ivol, double* rho, double* out, cudaStream_t st);
cudaError_t launch_plain_diag_gauss(const PlainYeeArgs& a, const double* rho, double rho_bg,
                                    double* out, cudaStream_t st);

}  // namespace pic
