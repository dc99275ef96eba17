// micro.cu -- initial conditions and microstructure generators, computed on the
// device in FP64 and handed to a problem through its ordinary field setters:
//   * crack / void initial condition (Eq. init_crack, Sec. 4.1.1) and the crack
//     in E, E = h(phi_init) E0 (Sec. 4.2.2);
//   * smooth random and two-phase Young's modulus fields (Sec. 3.3): low-pass
//     filter of caller-drawn white noise through the library's FFT passes, then
//     scaling and the algebraic sigmoid, or the sign and explicit Allen-Cahn
//     smoothing (Eq. ACsmooth), E = E0 xi.
// Readings (also used by the oracle): the support |r| <= 2 ell; "edge" notch =
// the printed r = (max(x - L/2, 0), y) with x in [-Lx/2, Lx/2) from the centre,
// "segment" = r = (max(|x| - L/2, 0), y); band 0 < |q| <= 2 pi / L_cut; sigmoid
// 1 - d D / (d^10 + D^10)^(1/10) below 1; population standard deviation.
#include <cmath>
#include <cstring>
#include <string>

#include "../../include/pff.h"
#include "kernels.cuh"
#include "launch.h"

namespace pff {
cudaError_t take_launch_error();   // launches rejected by the runtime on this host thread (or the last error)
namespace {

constexpr int MT = 256;

inline unsigned blocks_for(size_t n) { return (unsigned)std::min<size_t>((n + MT - 1) / MT, 4096); }

__global__ void k_crack_field(double* out, int nx, int ny, double dx, double ell, double xc, double yc, double len,
                              int shape, int modulus, double E0) {
    const size_t n = (size_t)nx * ny;
    const double Lx = nx * dx, Ly = ny * dx;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx), y = (int)(i / nx);
        double ddx = x * dx - xc, ddy = y * dx - yc;
        ddx -= Lx * floor(ddx / Lx + 0.5);   // nearest image, in [-Lx/2, Lx/2)
        ddy -= Ly * floor(ddy / Ly + 0.5);
        const double rx = shape == PFF_CRACK_SEGMENT ? fmax(fabs(ddx) - 0.5 * len, 0.0) : fmax(ddx - 0.5 * len, 0.0);
        const double r = sqrt(rx * rx + ddy * ddy);
        const double t = 1.0 - r / (2.0 * ell);
        const double phi = r <= 2.0 * ell ? t * t : 0.0;
        out[i] = modulus ? (1.0 - phi) * (1.0 - phi) * E0 : phi;
    }
}

// per-block sum and sum of squares (fixed tree), then one block totals them
__global__ void k_moments_part(const double* f, size_t n, double* part) {
    __shared__ double s1[MT], s2[MT];
    double a = 0.0, b = 0.0;
    for (size_t i = (size_t)blockIdx.x * MT + threadIdx.x; i < n; i += (size_t)gridDim.x * MT) {
        a += f[i];
        b += f[i] * f[i];
    }
    s1[threadIdx.x] = a;
    s2[threadIdx.x] = b;
    __syncthreads();
    for (int o = MT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) { s1[threadIdx.x] += s1[threadIdx.x + o]; s2[threadIdx.x] += s2[threadIdx.x + o]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) { part[2 * blockIdx.x] = s1[0]; part[2 * blockIdx.x + 1] = s2[0]; }
}

__global__ void k_moments_final(const double* part, int nb, size_t n, double* stats) {
    __shared__ double s1[MT], s2[MT];
    double a = 0.0, b = 0.0;
    for (int j = threadIdx.x; j < nb; j += MT) { a += part[2 * j]; b += part[2 * j + 1]; }
    s1[threadIdx.x] = a;
    s2[threadIdx.x] = b;
    __syncthreads();
    for (int o = MT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) { s1[threadIdx.x] += s1[threadIdx.x + o]; s2[threadIdx.x] += s2[threadIdx.x + o]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double mean = s1[0] / (double)n;
        const double var = fmax(s2[0] / (double)n - mean * mean, 0.0);
        stats[0] = mean;
        stats[1] = sqrt(var);
    }
}

// xi_r = f STD_t / STD(f) + 1, then the sigmoid floor below 1; E = E0 xi_r
__global__ void k_random_apply(const double* f, double* E, size_t n, const double* stats, double std_t, double xi_min,
                               double E0) {
    const double g = std_t / stats[1];
    const double D = 1.0 - xi_min, D10 = pow(D, 10.0);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        double xr = f[i] * g + 1.0;
        if (xr < 1.0) {
            const double d = 1.0 - xr;
            xr = 1.0 - d * D / pow(pow(d, 10.0) + D10, 0.1);
        }
        E[i] = E0 * xr;
    }
}

__global__ void k_sign(const double* f, double* out, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = (double)((f[i] > 0.0) - (f[i] < 0.0));
}

// one iteration of Eq. ACsmooth with the periodic 5-point stencil (pixel units)
__global__ void k_allen_cahn(const double* in, double* out, int nx, int ny) {
    const size_t n = (size_t)nx * ny;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx), y = (int)(i / nx);
        const double c = in[i];
        const double l = in[(size_t)y * nx + (x == 0 ? nx - 1 : x - 1)];
        const double r = in[(size_t)y * nx + (x == nx - 1 ? 0 : x + 1)];
        const double u = in[(size_t)(y == 0 ? ny - 1 : y - 1) * nx + x];
        const double dn = in[(size_t)(y == ny - 1 ? 0 : y + 1) * nx + x];
        const double lap5 = 4.0 * c - l - u - r - dn;
        out[i] = c - 0.1 * ((c * c * c - c) + lap5);
    }
}

__global__ void k_affine(const double* in, double* out, size_t n, double a, double b) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = a * in[i] + b;
}

}  // namespace

void micro_crack(double* out, int nx, int ny, double dx, double ell, double xc, double yc, double len, int shape,
                 int modulus, double E0, cudaStream_t st) {
    k_crack_field<<<blocks_for((size_t)nx * ny), MT, 0, st>>>(out, nx, ny, dx, ell, xc, yc, len, shape, modulus, E0);
    count_launch();
}

// E (device, FP64, nx*ny) from white noise (device, FP64) for the parameters mp.
// Scratch is allocated here and freed before returning (the call synchronises st).
int micro_generate(int nx, int ny, double dx, const pff_micro_params& mp, const double* noise_dev, double* E_dev,
                   const double2* tw64, cudaStream_t st, std::string& err) {
    const size_t n = (size_t)nx * ny;
    const int wp = ((nx / 2 + 1 + 15) / 16) * 16;
    const unsigned nb = blocks_for(n);
    double *a = nullptr, *b = nullptr, *part = nullptr, *stats = nullptr;
    double2* S = nullptr;
    Desc<double>* dd = nullptr;
    Ctrl* ctrl = nullptr;
    auto cleanup = [&]() {
        cudaFree(a); cudaFree(b); cudaFree(part); cudaFree(stats); cudaFree(S); cudaFree(dd); cudaFree(ctrl);
    };
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMalloc(&a, n * 8);
    if (e == cudaSuccess) e = cudaMalloc(&b, n * 8);
    if (e == cudaSuccess) e = cudaMalloc(&part, (size_t)2 * nb * 8);
    if (e == cudaSuccess) e = cudaMalloc(&stats, 2 * 8);
    if (e == cudaSuccess) e = cudaMalloc(&S, (size_t)ny * wp * sizeof(double2));
    if (e == cudaSuccess) e = cudaMalloc(&dd, sizeof(Desc<double>));
    if (e == cudaSuccess) e = cudaMalloc(&ctrl, sizeof(Ctrl));
    if (e != cudaSuccess) {
        cudaGetLastError();
        cleanup();
        err = "out of device memory for the generator scratch";
        return PFF_ERR_OOM;
    }
    Desc<double> h;
    std::memset(&h, 0, sizeof(h));
    h.r[0] = a;   // FCopyIn reads r[0]
    h.q[0] = b;   // FCopyOut writes q[0]
    h.S = S;
    h.tw = tw64;
    h.part = part;
    h.ctrl = ctrl;
    h.nx = nx;
    h.ny = ny;
    h.wp = wp;
    h.k.inv_n = 1.0 / ((double)nx * (double)ny);
    h.k.two_pi_over_Lx = 2.0 * M_PI / (nx * dx);
    h.k.two_pi_over_Ly = 2.0 * M_PI / (ny * dx);
    const double Lx = nx * dx, Ly = ny * dx;
    h.k.lp_a = (Ly * mp.L_cut) * (Ly * mp.L_cut);
    h.k.lp_b = (Lx * mp.L_cut) * (Lx * mp.L_cut);
    h.k.lp_c = (Lx * Ly) * (Lx * Ly);
    e = cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dd, &h, sizeof(h), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(a, noise_dev, n * 8, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) {
        launch_row_fwd<double>(RF_COPY1, nx, ny, dd, 1, st);
        launch_col<double>(CO_LOWPASS, nx, ny, wp, dd, 1, st);
        launch_row_inv<double>(RI_COPY1, nx, ny, dd, 1, st);   // b = filtered xi
        if (mp.kind == PFF_MICRO_RANDOM) {
            k_moments_part<<<nb, MT, 0, st>>>(b, n, part);
            k_moments_final<<<1, MT, 0, st>>>(part, (int)nb, n, stats);
            k_random_apply<<<nb, MT, 0, st>>>(b, E_dev, n, stats, mp.std_target, mp.xi_min, mp.E0);
            count_launch(); count_launch(); count_launch();
        } else {
            k_sign<<<nb, MT, 0, st>>>(b, a, n);
            count_launch();
            double* src = a;
            double* dst = b;
            for (int it = 0; it < mp.ac_iters; ++it) {
                k_allen_cahn<<<nb, MT, 0, st>>>(src, dst, nx, ny);
                count_launch();
                std::swap(src, dst);
            }
            k_affine<<<nb, MT, 0, st>>>(src, E_dev, n, mp.E0 * mp.a, mp.E0);
            count_launch();
        }
        e = take_launch_error();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cleanup();
    if (e != cudaSuccess) {
        err = std::string("microstructure generator: ") + cudaGetErrorString(e);
        return PFF_ERR_CUDA;
    }
    return PFF_OK;
}

}  // namespace pff
