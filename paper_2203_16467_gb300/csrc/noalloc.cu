// noalloc.cu -- pff_apply_laplacian_noalloc (FP64) and _f32: the collocation
// Laplacian of a caller-owned device field, computed without allocating memory.
//
// Some callers cannot call cudaMalloc: a framework that has reserved the whole
// device memory for its own pool, a latency-critical loop that cannot afford
// the implicit device synchronisation an allocation may cause, or a caller
// that must not leave allocations behind.  These entry points run the same
// three kernels as pff_apply_laplacian, but their scratch (one half spectrum of
// at most PFF_NOALLOC_MAX_N x (PFF_NOALLOC_MAX_N/2 + 16) complex values per
// precision, about 2.2 MB in FP64 and 1.1 MB in FP32), twiddle tables and
// kernel descriptors are file-scope device arrays that every GPU loading the
// library keeps until exit.
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/pff.h"
#include "kernels.cuh"

namespace pff {
cudaError_t take_launch_error();   // launches rejected by the runtime on this host thread
namespace {

constexpr int NA_MAX = PFF_NOALLOC_MAX_N;
constexpr int NA_WP = ((NA_MAX / 2 + 1 + 15) / 16) * 16;
constexpr int NA_TW = 2 * NA_MAX;   // twiddle tables for lengths up to NA_MAX

static __device__ __align__(256) double2 g_na_spectrum[(size_t)NA_MAX * NA_WP];
static __device__ __align__(256) double2 g_na_twiddles[NA_TW];
static __device__ __align__(256) Desc<double> g_na_desc;
static __device__ __align__(256) float2 g_na_spectrum_f[(size_t)NA_MAX * NA_WP];
static __device__ __align__(256) float2 g_na_twiddles_f[NA_TW];
static __device__ __align__(256) Desc<float> g_na_desc_f;

struct DeviceSymbols {
    bool ready = false;
    double2* spectrum = nullptr;
    double2* twiddles = nullptr;
    Desc<double>* desc = nullptr;
    float2* spectrum_f = nullptr;
    float2* twiddles_f = nullptr;
    Desc<float>* desc_f = nullptr;
};
constexpr int NA_MAX_DEVICES = 64;
DeviceSymbols g_symbols[NA_MAX_DEVICES];
std::mutex g_mu;

template <typename S>
bool symbol(const S& sym, void** p) {
    if (cudaGetSymbolAddress(p, sym) == cudaSuccess) return true;
    cudaGetLastError();
    return false;
}

// Once per device, with that device current: device addresses of the arrays
// (the names are host-side stand-ins in host code) and the twiddle tables.
int setup(int dev, DeviceSymbols& out, const char** msg) {
    std::lock_guard<std::mutex> g(g_mu);
    DeviceSymbols& s = g_symbols[dev];
    if (!s.ready) {
        void* p[6] = {};
        if (!symbol(g_na_spectrum, &p[0]) || !symbol(g_na_twiddles, &p[1]) || !symbol(g_na_desc, &p[2]) ||
            !symbol(g_na_spectrum_f, &p[3]) || !symbol(g_na_twiddles_f, &p[4]) || !symbol(g_na_desc_f, &p[5])) {
            *msg = "cudaGetSymbolAddress failed";
            return PFF_ERR_CUDA;
        }
        s.spectrum = (double2*)p[0];
        s.twiddles = (double2*)p[1];
        s.desc = (Desc<double>*)p[2];
        s.spectrum_f = (float2*)p[3];
        s.twiddles_f = (float2*)p[4];
        s.desc_f = (Desc<float>*)p[5];
        static double2 tw[NA_TW];   // host staging without a heap allocation
        static float2 twf[NA_TW];
        tw[0] = make_double2(1.0, 0.0);
        tw[1] = make_double2(1.0, 0.0);
        for (int M = 2; M <= NA_MAX; M *= 2)
            for (int j = 0; j < M; ++j) {
                double a = -2.0 * M_PI * (double)j / (double)M;
                tw[M + j] = make_double2(std::cos(a), std::sin(a));
            }
        for (int j = 0; j < NA_TW; ++j) twf[j] = make_float2((float)tw[j].x, (float)tw[j].y);
        // a copy from pageable memory may return before its DMA has landed, and kernels on
        // non-blocking streams do not wait for the legacy stream: the device synchronisation
        // makes the tables complete before any call can read them
        if (cudaMemcpyToSymbol(g_na_twiddles, tw, sizeof(double2) * NA_TW) != cudaSuccess ||
            cudaMemcpyToSymbol(g_na_twiddles_f, twf, sizeof(float2) * NA_TW) != cudaSuccess ||
            cudaDeviceSynchronize() != cudaSuccess) {
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

template <typename T, typename C, typename DS>
int apply(int nx, int ny, double dx, const T* in_dev, T* out_dev, void* cuda_stream, const char** err_msg,
          C* spectrum, C* twiddles, Desc<T>* desc_dev, const DS& desc_sym) {
    const char* dummy = nullptr;
    const char** msg = err_msg ? err_msg : &dummy;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    Desc<T> d;
    std::memset(&d, 0, sizeof(d));
    d.r[0] = const_cast<T*>(in_dev);   // FCopyIn reads r[0]
    d.q[0] = out_dev;                  // FCopyOut writes q[0]
    d.S = spectrum;
    d.tw = twiddles;
    d.nx = nx;
    d.ny = ny;
    d.wp = ((nx / 2 + 1 + 15) / 16) * 16;
    d.k.inv_n = 1.0 / ((double)nx * (double)ny);
    d.k.two_pi_over_Lx = 2.0 * M_PI / (nx * dx);
    d.k.two_pi_over_Ly = 2.0 * M_PI / (ny * dx);
    // pageable source: the copy has left d before this call returns
    if (cudaMemcpyToSymbolAsync(desc_sym, &d, sizeof(d), 0, cudaMemcpyHostToDevice, st) != cudaSuccess) {
        cudaGetLastError();
        *msg = "descriptor upload failed";
        return PFF_ERR_CUDA;
    }
    launch_row_fwd<T>(RF_COPY1, nx, ny, desc_dev, 1, st);
    launch_col<T>(CO_LAP_PLAIN, nx, ny, d.wp, desc_dev, 1, st);
    launch_row_inv<T>(RI_COPY1, nx, ny, desc_dev, 1, st);
    if (take_launch_error() != cudaSuccess) {
        *msg = "kernel launch failed";
        return PFF_ERR_CUDA;
    }
    return PFF_OK;
}

int check(int nx, int ny, double dx, const void* in_dev, const void* out_dev, const char** msg,
          DeviceSymbols& sym) {
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
    return setup(dev, sym, msg);
}

}  // namespace
}  // namespace pff

extern "C" int pff_apply_laplacian_noalloc(int nx, int ny, double dx, const double* in_dev, double* out_dev,
                                           void* cuda_stream, const char** err_msg) {
    using namespace pff;
    const char* dummy = nullptr;
    const char** msg = err_msg ? err_msg : &dummy;
    *msg = nullptr;
    DeviceSymbols sym;
    int rc = check(nx, ny, dx, in_dev, out_dev, msg, sym);
    if (rc) return rc;
    return apply<double>(nx, ny, dx, in_dev, out_dev, cuda_stream, msg, sym.spectrum, sym.twiddles, sym.desc,
                         g_na_desc);
}

extern "C" int pff_apply_laplacian_noalloc_f32(int nx, int ny, double dx, const float* in_dev, float* out_dev,
                                               void* cuda_stream, const char** err_msg) {
    using namespace pff;
    const char* dummy = nullptr;
    const char** msg = err_msg ? err_msg : &dummy;
    *msg = nullptr;
    DeviceSymbols sym;
    int rc = check(nx, ny, dx, in_dev, out_dev, msg, sym);
    if (rc) return rc;
    return apply<float>(nx, ny, dx, in_dev, out_dev, cuda_stream, msg, sym.spectrum_f, sym.twiddles_f,
                        sym.desc_f, g_na_desc_f);
}
