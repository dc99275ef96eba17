// noalloc.cu -- pff_apply_laplacian_noalloc: the collocation Laplacian of a
// caller-owned FP64 device field, computed without allocating any memory.
//
// Some callers cannot call cudaMalloc: a framework that has reserved the whole
// device memory for its own pool, a latency-critical loop that cannot afford
// the implicit device synchronisation an allocation may cause, or a caller
// that must not leave allocations behind.  This entry point runs the same
// three kernels as pff_apply_laplacian, but its scratch (one half spectrum of
// at most PFF_NOALLOC_MAX_N x (PFF_NOALLOC_MAX_N/2 + 16) complex FP64 values,
// about 2.2 MB), its twiddle table and its kernel descriptor are file-scope
// device arrays that every GPU loading the library keeps until exit.
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/pff.h"
#include "kernels.cuh"

namespace pff {
namespace {

constexpr int NA_MAX = PFF_NOALLOC_MAX_N;
constexpr int NA_WP = ((NA_MAX / 2 + 1 + 15) / 16) * 16;
constexpr int NA_TW = 2 * NA_MAX;   // twiddle tables for lengths up to NA_MAX

static __device__ __align__(256) double2 g_na_spectrum[(size_t)NA_MAX * NA_WP];
static __device__ __align__(256) double2 g_na_twiddles[NA_TW];
static __device__ __align__(256) Desc<double> g_na_desc;

struct DeviceSymbols {
    bool ready = false;
    double2* spectrum = nullptr;
    double2* twiddles = nullptr;
    Desc<double>* desc = nullptr;
};
constexpr int NA_MAX_DEVICES = 64;
DeviceSymbols g_symbols[NA_MAX_DEVICES];
std::mutex g_mu;

// Once per device, with that device current: device addresses of the arrays
// (the names are host-side stand-ins in host code) and the twiddle table.
int setup(int dev, DeviceSymbols& out, const char** msg) {
    std::lock_guard<std::mutex> g(g_mu);
    DeviceSymbols& s = g_symbols[dev];
    if (!s.ready) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_na_spectrum) != cudaSuccess) { *msg = "cudaGetSymbolAddress(spectrum) failed"; cudaGetLastError(); return PFF_ERR_CUDA; }
        s.spectrum = (double2*)p;
        if (cudaGetSymbolAddress(&p, g_na_twiddles) != cudaSuccess) { *msg = "cudaGetSymbolAddress(twiddles) failed"; cudaGetLastError(); return PFF_ERR_CUDA; }
        s.twiddles = (double2*)p;
        if (cudaGetSymbolAddress(&p, g_na_desc) != cudaSuccess) { *msg = "cudaGetSymbolAddress(descriptor) failed"; cudaGetLastError(); return PFF_ERR_CUDA; }
        s.desc = (Desc<double>*)p;
        static double2 tw[NA_TW];   // host staging without a heap allocation
        tw[0] = make_double2(1.0, 0.0);
        tw[1] = make_double2(1.0, 0.0);
        for (int M = 2; M <= NA_MAX; M *= 2)
            for (int j = 0; j < M; ++j) {
                double a = -2.0 * M_PI * (double)j / (double)M;
                tw[M + j] = make_double2(std::cos(a), std::sin(a));
            }
        if (cudaMemcpyToSymbol(g_na_twiddles, tw, sizeof(double2) * NA_TW) != cudaSuccess) {
            *msg = "twiddle upload failed";
            cudaGetLastError();
            return PFF_ERR_CUDA;
        }
        s.ready = true;
    }
    out = s;
    return PFF_OK;
}

bool pow2_in_range(int n) { return n >= 16 && n <= NA_MAX && (n & (n - 1)) == 0; }

}  // namespace
}  // namespace pff

extern "C" int pff_apply_laplacian_noalloc(int nx, int ny, double dx, const double* in_dev, double* out_dev,
                                           void* cuda_stream, const char** err_msg) {
    using namespace pff;
    const char* dummy = nullptr;
    const char** msg = err_msg ? err_msg : &dummy;
    *msg = nullptr;
    if (!pow2_in_range(nx) || !pow2_in_range(ny)) {
        *msg = "nx and ny must be powers of two from 16 to PFF_NOALLOC_MAX_N (512)";
        return PFF_ERR_INVALID_ARG;
    }
    if (!(dx > 0.0) || !in_dev || !out_dev) {
        *msg = "dx must be positive and both device pointers non-null";
        return PFF_ERR_INVALID_ARG;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
        cudaGetLastError();
        *msg = "no usable current CUDA device";
        return PFF_ERR_CUDA;
    }
    DeviceSymbols sym;
    int rc = setup(dev, sym, msg);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    Desc<double> d;
    std::memset(&d, 0, sizeof(d));
    d.r[0] = const_cast<double*>(in_dev);   // FCopyIn reads r[0]
    d.q[0] = out_dev;                       // FCopyOut writes q[0]
    d.S = sym.spectrum;
    d.tw = sym.twiddles;
    d.nx = nx;
    d.ny = ny;
    d.wp = ((nx / 2 + 1 + 15) / 16) * 16;
    d.k.inv_n = 1.0 / ((double)nx * (double)ny);
    d.k.two_pi_over_Lx = 2.0 * M_PI / (nx * dx);
    d.k.two_pi_over_Ly = 2.0 * M_PI / (ny * dx);
    // pageable source: the copy has left d before this call returns
    if (cudaMemcpyToSymbolAsync(g_na_desc, &d, sizeof(d), 0, cudaMemcpyHostToDevice, st) != cudaSuccess) {
        cudaGetLastError();
        *msg = "descriptor upload failed";
        return PFF_ERR_CUDA;
    }
    launch_row_fwd<double>(RF_COPY1, nx, ny, sym.desc, 1, st);
    launch_col<double>(CO_LAP_PLAIN, nx, ny, d.wp, sym.desc, 1, st);
    launch_row_inv<double>(RI_COPY1, nx, ny, sym.desc, 1, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        *msg = "kernel launch failed";
        return PFF_ERR_CUDA;
    }
    return PFF_OK;
}
