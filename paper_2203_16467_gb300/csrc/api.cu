// api.cu -- C ABI of libpff (include/pff.h): problem state, parameter
// resolution, the host-side loop of one load step (Algorithm 4) over a group
// of problems of equal size and precision, batching, and field I/O.
//
// The host only sequences kernels.  Every solver scalar (CG / BCCG step
// lengths, convergence flags, the rescale factor, the strain increment) is
// computed and consumed on the device; the host polls the per-problem done
// flags once per chunk of iterations.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "../../include/pff.h"
#include "common.cuh"
#include "launch.h"

namespace pff {

static std::atomic<unsigned long long> g_launches{0};
static thread_local bool t_capturing = false;   // this thread is capturing a graph
void count_launch() {
    if (!t_capturing) g_launches.fetch_add(1, std::memory_order_relaxed);
}

// ---- per-kernel-class event timing
struct TimingState {
    std::mutex mu;
    bool on = false;
    std::vector<cudaEvent_t> pool;
    struct Pending { int key; cudaEvent_t a, b; };
    std::vector<Pending> pending;
    std::map<int, std::pair<double, unsigned long long>> acc;
};
static TimingState g_tm;
static thread_local std::map<int, cudaEvent_t> t_open;   // begin events of this host thread
bool timing_on() { return g_tm.on; }

// programmatic dependent launch of the operator kernels (off while timing: the
// per-kernel events need each kernel to start after its predecessor completed)
static std::atomic<bool> g_pdl{true};
// (inside captured graphs programmatic edges measured slower than plain kernel
// edges, so only direct launches use it)
bool pdl_on() { return g_pdl.load(std::memory_order_relaxed) && !g_tm.on && !t_capturing; }
static cudaEvent_t tm_event() {
    if (!g_tm.pool.empty()) { cudaEvent_t e = g_tm.pool.back(); g_tm.pool.pop_back(); return e; }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}
void timing_begin(int key, cudaStream_t st) {
    std::lock_guard<std::mutex> g(g_tm.mu);
    cudaEvent_t e = tm_event();
    cudaEventRecord(e, st);
    t_open[key] = e;
}
void timing_end(int key, cudaStream_t st) {
    std::lock_guard<std::mutex> g(g_tm.mu);
    auto it = t_open.find(key);
    if (it == t_open.end()) return;
    cudaEvent_t e = tm_event();
    cudaEventRecord(e, st);
    g_tm.pending.push_back({key, it->second, e});
    t_open.erase(it);
}
// fold completed event pairs into the totals (caller has synchronized the streams)
static void timing_collect() {
    std::lock_guard<std::mutex> g(g_tm.mu);
    std::vector<TimingState::Pending> keep;
    for (auto& p : g_tm.pending) {
        float ms = 0.f;
        if (cudaEventQuery(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            auto& a = g_tm.acc[p.key];
            a.first += ms;
            a.second += 1;
            g_tm.pool.push_back(p.a);
            g_tm.pool.push_back(p.b);
        } else {
            keep.push_back(p);
        }
    }
    cudaGetLastError();
    g_tm.pending.swap(keep);
}

void note_launch_error(cudaError_t e);
// FFT shape variants: columns per block of the 512-point FP32 column pass, for one (index 0) and
// three (index 1) components; a change bumps the generation, and graph caches captured with
// another generation are re-captured
static std::atomic<int> g_col512_cw[2] = {{4}, {4}};
static std::atomic<int> g_shape_gen{0};
// BCCG iteration structure: three passes (alpha from the column pass, iterate fused into the
// J p pass; default) or the four-pass chain of the preconditioned variant (alpha from p.Jp)
static std::atomic<bool> g_bccg4{false};
int col512_cw(int nc);
// Opt a kernel in to its dynamic shared memory when static plus dynamic shared
// memory exceeds the 48 KB available without the attribute.
int col512_cw(int nc) { return g_col512_cw[nc == 3 ? 1 : 0].load(std::memory_order_relaxed); }

bool smem_optin(const void* fn, size_t smem) {
    int dev = 0;
    cudaGetDevice(&dev);
    static std::mutex mu;
    static std::unordered_map<const void*, unsigned long long> done;
    std::lock_guard<std::mutex> g(mu);
    unsigned long long& m = done[fn];
    if (m & (1ull << (dev & 63))) return true;
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, fn);
    if (e == cudaSuccess && fa.sharedSizeBytes + smem > 48 * 1024)
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) m |= 1ull << (dev & 63);
    else note_launch_error(e);
    return e == cudaSuccess;
}

// The first failed launch of this host thread, reported by the next poll of the
// group (kernel launches return configuration errors only to their caller).
static thread_local cudaError_t t_launch_err = cudaSuccess;
void note_launch_error(cudaError_t e) {
    if (t_launch_err == cudaSuccess) t_launch_err = e;
}
cudaError_t take_launch_error() {
    cudaError_t e = t_launch_err;
    t_launch_err = cudaSuccess;
    if (e == cudaSuccess) e = cudaGetLastError();
    return e;
}

// Keeps the stream busy for about ns nanoseconds (bounded by time and by an
// iteration cap; it waits on nothing).  Used only in timing mode, so that the
// host queues a whole chunk of launches before the first one starts and the
// event brackets measure device time rather than host submission gaps.
__global__ void k_delay(unsigned long long ns) {
    if (threadIdx.x != 0) return;
    unsigned long long t0, t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (int it = 0; it < (1 << 24); ++it) {
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 >= ns) break;
    }
}

__global__ void k_d2f(float* dst, const double* src, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = (float)src[i];
}
__global__ void k_f2d(double* dst, const float* src, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = (double)src[i];
}
void launch_convert_d2f(float* dst, const double* src, size_t n, cudaStream_t st) {
    k_d2f<<<(unsigned)std::min<size_t>((n + 255) / 256, 4096), 256, 0, st>>>(dst, src, n);
    count_launch();
}
void launch_convert_f2d(double* dst, const float* src, size_t n, cudaStream_t st) {
    k_f2d<<<(unsigned)std::min<size_t>((n + 255) / 256, 4096), 256, 0, st>>>(dst, src, n);
    count_launch();
}

// Twiddle tables, one pair per device: entry M + j = exp(-2 pi i j / M) for
// every power of two M <= TW_MAX (computed in FP64 on the host).
struct Twiddles {
    float2* t32 = nullptr;
    double2* t64 = nullptr;
};
// k_persist.cu
int persist_bccg_blocks(int share_den);
cudaError_t launch_persist_bccg(const Desc<float>* d, int max_iters, int blocks, cudaStream_t st);
void persist_set_spin(long long cycles);
// micro.cu
void micro_crack(double* out, int nx, int ny, double dx, double ell, double xc, double yc, double len, int shape,
                 int modulus, double E0, cudaStream_t st);
int micro_generate(int nx, int ny, double dx, const pff_micro_params& mp, const double* noise_dev, double* E_dev,
                   const double2* tw64, cudaStream_t st, std::string& err);
static const int TWN = 4096;
static int twiddles_for(int dev, Twiddles& out) {
    static std::mutex mu;
    static std::map<int, Twiddles> tabs;
    std::lock_guard<std::mutex> g(mu);
    auto it = tabs.find(dev);
    if (it != tabs.end()) { out = it->second; return 0; }
    std::vector<double2> h64(2 * TWN);
    std::vector<float2> h32(2 * TWN);
    h64[0] = make_double2(1.0, 0.0);
    h64[1] = make_double2(1.0, 0.0);
    for (int M = 2; M <= TWN; M *= 2)
        for (int j = 0; j < M; ++j) {
            double a = -2.0 * M_PI * (double)j / (double)M;
            h64[M + j] = make_double2(std::cos(a), std::sin(a));
        }
    for (int i = 0; i < 2 * TWN; ++i) h32[i] = make_float2((float)h64[i].x, (float)h64[i].y);
    Twiddles t;
    if (cudaMalloc(&t.t32, sizeof(float2) * 2 * TWN) != cudaSuccess) return -1;
    if (cudaMalloc(&t.t64, sizeof(double2) * 2 * TWN) != cudaSuccess) { cudaFree(t.t32); return -1; }
    // pageable sources: the device synchronisation makes the tables complete before kernels
    // on any (non-blocking) stream can read them
    if (cudaMemcpy(t.t32, h32.data(), sizeof(float2) * 2 * TWN, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(t.t64, h64.data(), sizeof(double2) * 2 * TWN, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess) {
        cudaFree(t.t32);
        cudaFree(t.t64);
        cudaGetLastError();
        return -1;
    }
    tabs[dev] = t;
    out = t;
    return 0;
}

static inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr int NFIELDS = 19;   // E, phi, eps*3, th*3, r*3, p*3, q*3, lap, aux
constexpr int PART_BLOCKS = 2048;
static int wp_of(int nx) { return ((nx / 2 + 1 + 15) / 16) * 16; }

static size_t problem_bytes(int nx, int ny, int prec) {
    size_t n = (size_t)nx * ny;
    size_t es = prec == PFF_FP64 ? 8 : 4;
    size_t b = NFIELDS * align256(n * es);
    b += align256(n);                                              // flags
    b += align256((size_t)3 * ny * wp_of(nx) * 2 * es);            // spectrum
    b += align256((size_t)PART_BLOCKS * 8 * sizeof(double));       // partials
    if (prec != PFF_FP64) b += align256(n * sizeof(double));       // FP64 staging of host transfers
    b += align256(sizeof(Ctrl));
    return b;
}

static bool valid_n(int n) { return n >= 16 && n <= 2048 && (n & (n - 1)) == 0; }

// CUDA graphs of the two fixed launch sequences of a load step (a chunk of CG
// iterations, a chunk of BCCG iterations), captured once per group shape.
struct GraphCache {
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    int nodes[2] = {0, 0};
    bool failed[2] = {false, false};   // capture or instantiation failed: launch directly
    const void* desc = nullptr;
    int np = 0;
    int cond = -1;                     // conditional-node setting the graphs were captured with
    int precond = -1;                  // preconditioner setting the graphs were captured with
    int gen = -1;                      // FFT shape generation the graphs were captured with
    void reset() {
        for (int k = 0; k < 2; ++k) {
            if (exec[k]) cudaGraphExecDestroy(exec[k]);
            exec[k] = nullptr;
            nodes[k] = 0;
            failed[k] = false;
        }
    }
};


}  // namespace pff

using namespace pff;

struct pff_problem {
    int nx = 0, ny = 0, prec = 0, wp = 0, dev = 0;
    cudaStream_t st = nullptr;
    pff_params prm{};
    int fracture = PFF_AT1, split = PFF_SPECTRAL, irrev = PFF_CRACK_SET;
    std::string err;
    char* base = nullptr;
    void* field[NFIELDS] = {};
    uint8_t* flags = nullptr;
    void* S = nullptr;
    double* stage = nullptr;       // FP64 staging for host transfers of FP32 fields (n values; FP32 problems)
    double* part = nullptr;
    Ctrl* ctrl = nullptr;
    Twiddles tw;
    void* d_desc = nullptr;        // Desc<T> of this problem alone
    int* d_flags = nullptr;        // group-of-one poll buffer
    Ctrl* d_ctrlcopy = nullptr;
    int* h_flags = nullptr;        // pinned
    Ctrl* h_ctrl = nullptr;        // pinned
    pff::GraphCache graphs;
    double td_dt = -1.0;           // time-dependent method: current time step (units of t~)
    double sumE = 0.0, sumE2 = 0.0;
    bool broken = false;
    int flag_host = 0;
    size_t bytes = 0;
    size_t n() const { return (size_t)nx * ny; }
};

namespace pff {

static int fail(pff_problem* h, int code, const std::string& msg) {
    if (h) h->err = msg;
    return code;
}
static int cuda_fail(pff_problem* h, cudaError_t e, const char* where) {
    return fail(h, PFF_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

static Consts make_consts(const pff_problem* h) {
    const pff_params& p = h->prm;
    Consts k{};
    double nu = p.nu;
    k.lam_c = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    k.mu_c = 1.0 / (2.0 * (1.0 + nu));
    double cw = h->fracture == PFF_AT1 ? 8.0 / 3.0 : 2.0;
    k.c = p.Gc / (cw * p.ell);
    k.kappa = 2.0 * k.c * p.ell * p.ell;
    k.ell2 = p.ell * p.ell;
    k.eta_dt = p.eta_over_dt >= 0.0 ? p.eta_over_dt : std::ldexp(1.0, -16) * p.Gc / p.ell;
    k.cf2 = k.c * (h->fracture == PFF_AT1 ? 0.0 : 2.0);
    k.Fmax = p.F_max >= 0.0 ? p.F_max : 0.7 * p.Gc / p.ell;
    k.thresh = p.thresh >= 0.0 ? p.thresh : 1.0 * p.Gc / p.ell;
    k.dphi_min = p.dphi_min;
    double meanE = h->sumE / (double)h->n();
    k.C_broken = p.C_broken > 0.0 ? p.C_broken : 0.01 * meanE;
    k.crack_thr = p.crack_set_threshold;
    const bool mixed = h->prec == PFF_MIXED;
    // FP32 fields carry ~1e-7 relative rounding: tolerances below these floors
    // cannot be observed on explicitly recomputed residuals.
    k.mech_tol = mixed ? std::max(p.mech_tol, 1e-6) : p.mech_tol;
    k.mech_cg_rtol = p.mech_cg_rtol;
    k.pf_tol = p.pf_tol;
    k.pf_atol = p.pf_atol;
    k.pf_floor = 0.0;
    for (int j = 0; j < 3; ++j) k.d_eps_bar[j] = p.d_eps_bar[j];
    k.dA = p.dx * p.dx;
    k.inv_n = 1.0 / (double)h->n();
    k.L1_scale = (p.dx / p.ell) * (p.dx / p.ell);
    k.two_pi_over_Lx = 2.0 * M_PI / (h->nx * p.dx);
    k.two_pi_over_Ly = 2.0 * M_PI / (h->ny * p.dx);
    k.max_newton = p.mech_max_newton;
    k.max_cg = p.mech_max_cg;
    k.max_pf = p.pf_max_iter;
    k.pf_precond = p.pf_precondition != 0;
    k.fracture = h->fracture;
    k.split = h->split;
    k.irrev = h->irrev;
    return k;
}

template <typename T>
static Desc<T> make_desc(const pff_problem* h) {
    Desc<T> d{};
    T** f = (T**)h->field;
    d.E = f[0];
    d.phi = f[1];
    for (int j = 0; j < 3; ++j) {
        d.eps[j] = f[2 + j];
        d.th[j] = f[5 + j];
        d.r[j] = f[8 + j];
        d.p[j] = f[11 + j];
        d.q[j] = f[14 + j];
    }
    d.lap = f[17];
    d.aux = f[18];
    d.flags = h->flags;
    d.S = (typename CT<T>::t*)h->S;
    if constexpr (sizeof(T) == 8) d.tw = h->tw.t64; else d.tw = h->tw.t32;
    d.part = h->part;
    d.ctrl = h->ctrl;
    d.nx = h->nx;
    d.ny = h->ny;
    d.wp = h->wp;
    d.k = make_consts(h);
    return d;
}

static int upload_desc(pff_problem* h) {
    cudaError_t e;
    if (h->prec == PFF_FP64) {
        Desc<double> d = make_desc<double>(h);
        e = cudaMemcpyAsync(h->d_desc, &d, sizeof(d), cudaMemcpyHostToDevice, h->st);
    } else {
        Desc<float> d = make_desc<float>(h);
        e = cudaMemcpyAsync(h->d_desc, &d, sizeof(d), cudaMemcpyHostToDevice, h->st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    return e == cudaSuccess ? 0 : cuda_fail(h, e, "upload descriptor");
}

// FP32 problems hold a staging buffer of n doubles (part of the problem's allocation) through
// which host transfers of their fields pass: the FP64 host values are copied as they are and
// converted on the device (and back), so a transfer is one DMA of the caller's buffer (fast
// when it is page-locked) and one kernel, with no conversion loop on the host.
static bool ensure_stage(pff_problem* h) { return h->stage != nullptr; }

// Copy nx*ny FP64 values (host or device) into a field of the problem's precision.
static int put_field(pff_problem* h, void* dst, const double* src, size_t count, int on_device) {
    cudaError_t e = cudaSuccess;
    if (h->prec == PFF_FP64) {
        e = cudaMemcpyAsync(dst, src, count * 8, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->st);
    } else if (on_device) {
        launch_convert_d2f((float*)dst, src, count, h->st);
        e = cudaGetLastError();
    } else if (count <= h->n() && ensure_stage(h)) {
        e = cudaMemcpyAsync(h->stage, src, count * 8, cudaMemcpyHostToDevice, h->st);
        if (e == cudaSuccess) {
            launch_convert_d2f((float*)dst, h->stage, count, h->st);
            e = cudaGetLastError();
        }
    } else {   // no room for the staging buffer: convert on the host
        std::vector<float> tmp(count);
        for (size_t i = 0; i < count; ++i) tmp[i] = (float)src[i];
        e = cudaMemcpyAsync(dst, tmp.data(), count * 4, cudaMemcpyHostToDevice, h->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);   // the caller may reuse its buffer on return
    return e == cudaSuccess ? 0 : cuda_fail(h, e, "copy in");
}

static int get_field(pff_problem* h, const void* src, double* dst, size_t count) {
    cudaError_t e;
    if (h->prec == PFF_FP64) {
        e = cudaMemcpyAsync(dst, src, count * 8, cudaMemcpyDeviceToHost, h->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    } else if (count <= h->n() && ensure_stage(h)) {
        launch_convert_f2d(h->stage, (const float*)src, count, h->st);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(dst, h->stage, count * 8, cudaMemcpyDeviceToHost, h->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    } else {
        std::vector<float> tmp(count);
        e = cudaMemcpyAsync(tmp.data(), src, count * 4, cudaMemcpyDeviceToHost, h->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
        for (size_t i = 0; i < count; ++i) dst[i] = (double)tmp[i];
    }
    return e == cudaSuccess ? 0 : cuda_fail(h, e, "copy out");
}

static int read_ctrl(pff_problem* h) {
    cudaError_t e = cudaMemcpyAsync(h->h_ctrl, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    return e == cudaSuccess ? 0 : cuda_fail(h, e, "read control block");
}
static int write_ctrl(pff_problem* h) {
    cudaError_t e = cudaMemcpyAsync(h->ctrl, h->h_ctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    return e == cudaSuccess ? 0 : cuda_fail(h, e, "write control block");
}

// ---------------------------------------------------------------------------
// A group: problems of equal (nx, ny, precision) whose kernels share launches.
struct Group {
    int nx, ny, wp, prec, np;
    cudaStream_t st;
    void* d_desc;          // Desc<T>[np]
    int* d_flags;          // np
    Ctrl* d_ctrl;          // np
    int* h_flags;          // pinned np
    Ctrl* h_ctrl;          // pinned np
    GraphCache* graphs;    // may be null (no graphs)
    int precond = 0;       // BCCG with the Fourier Helmholtz preconditioner (same for all problems)
};

static const int CHUNK = 12;
static bool g_graphs_enabled = true;
static bool g_cond_nodes = false;  // BCCG explicit-residual chain in conditional graph nodes
static bool g_persist = false;     // persistent BCCG solve for single FP32 512^2 problems (opt-in)
static std::atomic<bool> g_cluster{false};  // cluster Newton-CG solve for FP32 512^2 problems (opt-in)

// The mechanics solve of a group in one cluster launch (FP32 512 x 512 problems),
// when enabled and the device can host it; returns false when the caller must
// run the per-kernel path instead.
template <typename T>
static bool mech_cluster_group(const Group& g) {
    if constexpr (sizeof(T) == 4) {
        if (!g_cluster.load() || g.nx != 512 || g.ny != 512 || !mech_cluster_supported()) return false;
        const bool tm = timing_on();   // kernel-class key: family 4 (cluster), op 0
        if (tm) timing_begin(4 * 16 + 0, g.st);
        cudaError_t e = launch_mech_cluster((const Desc<float>*)g.d_desc, g.np, g.st);
        if (tm) timing_end(4 * 16 + 0, g.st);
        if (e != cudaSuccess) {   // not launched: the per-kernel path runs instead
            cudaGetLastError();
            return false;
        }
        return true;
    } else {
        (void)g;
        return false;
    }
}
static int g_persist_share = 8;    // the persistent launch takes 1/share of the resident capacity

template <typename T>
static void chunk_direct(int kind, const Group& g) {
    const Desc<T>* d = (const Desc<T>*)g.d_desc;
    const int nx = g.nx, ny = g.ny, wp = g.wp, np = g.np;
    cudaStream_t st = g.st;
    for (int c = 0; c < CHUNK; ++c) {
        if (kind == 0) {
            launch_row_fwd<T>(RF_CG, nx, ny, d, np, st);
            launch_col<T>(CO_GAMMA_CG, nx, ny, wp, d, np, st);
            launch_row_inv<T>(RI_CG, nx, ny, d, np, st);
        } else {
            if (g.precond) {   // z = M^-1 r on the free set, beta
                launch_row_fwd<T>(RF_PF_Z, nx, ny, d, np, st);
                launch_col<T>(CO_PRECOND, nx, ny, wp, d, np, st);
                launch_row_inv<T>(RI_PF_Z, nx, ny, d, np, st);
            }
            if (g.precond || g_bccg4.load()) {
                launch_row_fwd<T>(RF_PF_A, nx, ny, d, np, st);
                launch_col<T>(CO_LAP_PF, nx, ny, wp, d, np, st);
                launch_row_inv<T>(RI_PF_A, nx, ny, d, np, st);
                launch_elem<T>(EL_PF_B, nx, ny, d, np, st);
            } else {   // alpha from the column pass, the iterate fused into the J p pass
                launch_row_fwd<T>(RF_PF_A, nx, ny, d, np, st);
                launch_col<T>(CO_LAP_PFQ, nx, ny, wp, d, np, st);
                launch_row_inv<T>(RI_PF_AB, nx, ny, d, np, st);
            }
            launch_row_fwd<T>(RF_PF_B, nx, ny, d, np, st);          // only when J v is evaluated
            launch_col<T>(CO_LAP_PF_FULL, nx, ny, wp, d, np, st);   // explicitly this iteration
            launch_row_inv<T>(RI_PF_B, nx, ny, d, np, st);
        }
    }
}

// Capture of a BCCG chunk in which the explicit J v - b chain of each iteration
// sits in a conditional (IF) graph node: a one-thread kernel sets the condition
// from the problems' pf_full flags, so iterations that take the residual by
// recurrence launch no kernels for the chain.
static cudaStream_t side_stream() {
    static thread_local std::map<int, cudaStream_t> side;
    int dev = 0;
    cudaGetDevice(&dev);
    auto it = side.find(dev);
    if (it != side.end()) return it->second;
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
    side[dev] = s;
    return s;
}

template <typename T>
static cudaError_t capture_pf_chunk(const Group& g, cudaGraph_t* out, int* kernels) {
    const Desc<T>* d = (const Desc<T>*)g.d_desc;
    const int nx = g.nx, ny = g.ny, wp = g.wp, np = g.np;
    cudaStream_t st = g.st, sd = side_stream();
    if (!sd) return cudaErrorNotSupported;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaGraphCreate(&graph, 0);
    if (e != cudaSuccess) return e;
    cudaGraphConditionalHandle h;
    if ((e = cudaGraphConditionalHandleCreate(&h, graph, 0, 0)) != cudaSuccess) { cudaGraphDestroy(graph); return e; }
    if ((e = cudaStreamBeginCaptureToGraph(st, graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
        cudaSuccess) {
        cudaGraphDestroy(graph);
        return e;
    }
    int nk = 0;
    for (int c = 0; c < CHUNK && e == cudaSuccess; ++c) {
        if (g.precond) {
            launch_row_fwd<T>(RF_PF_Z, nx, ny, d, np, st);
            launch_col<T>(CO_PRECOND, nx, ny, wp, d, np, st);
            launch_row_inv<T>(RI_PF_Z, nx, ny, d, np, st);
            nk += 3;
        }
        if (g.precond || g_bccg4.load()) {
            launch_row_fwd<T>(RF_PF_A, nx, ny, d, np, st);
            launch_col<T>(CO_LAP_PF, nx, ny, wp, d, np, st);
            launch_row_inv<T>(RI_PF_A, nx, ny, d, np, st);
            launch_elem<T>(EL_PF_B, nx, ny, d, np, st);
            nk += 4;
        } else {
            launch_row_fwd<T>(RF_PF_A, nx, ny, d, np, st);
            launch_col<T>(CO_LAP_PFQ, nx, ny, wp, d, np, st);
            launch_row_inv<T>(RI_PF_AB, nx, ny, d, np, st);
            nk += 3;
        }
        launch_pf_cond<T>(d, np, h, st);
        nk += 1;
        cudaStreamCaptureStatus cs;
        const cudaGraphNode_t* deps = nullptr;
        size_t nd = 0;
        if ((e = cudaStreamGetCaptureInfo(st, &cs, nullptr, nullptr, &deps, nullptr, &nd)) != cudaSuccess) break;
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeIf;
        cp.conditional.size = 1;
        cudaGraphNode_t node;
        if ((e = cudaGraphAddNode(&node, graph, deps, nullptr, nd, &cp)) != cudaSuccess) break;
        if ((e = cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies)) !=
            cudaSuccess)
            break;
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        if ((e = cudaStreamBeginCaptureToGraph(sd, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
            cudaSuccess)
            break;
        launch_row_fwd<T>(RF_PF_B, nx, ny, d, np, sd);
        launch_col<T>(CO_LAP_PF_FULL, nx, ny, wp, d, np, sd);
        launch_row_inv<T>(RI_PF_B, nx, ny, d, np, sd);
        cudaGraph_t body_out = nullptr;
        if ((e = cudaStreamEndCapture(sd, &body_out)) != cudaSuccess) break;
    }
    cudaGraph_t done = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(st, &done);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return e;
    }
    *out = graph;
    *kernels = nk;
    return cudaSuccess;
}

// One chunk of iterations: replayed from a captured graph when the group has a
// graph cache and a non-default stream, and timing is off; launched directly otherwise.
template <typename T>
static void run_chunk(int kind, Group& g, bool& warmed) {
    GraphCache* gc = g.graphs;
    if (timing_on()) {
        k_delay<<<1, 32, 0, g.st>>>(kind == 0 ? 400000ull : 600000ull);
        chunk_direct<T>(kind, g);
        warmed = true;
        return;
    }
    if (!gc || !g_graphs_enabled || g.st == nullptr || !warmed) {
        chunk_direct<T>(kind, g);
        warmed = true;   // attributes (shared-memory opt-in) are set by the first direct chunk
        return;
    }
    if (gc->desc != g.d_desc || gc->np != g.np || gc->cond != (int)g_cond_nodes || gc->precond != g.precond ||
        gc->gen != g_shape_gen.load()) {
        gc->reset();
        gc->desc = g.d_desc;
        gc->np = g.np;
        gc->cond = (int)g_cond_nodes;
        gc->precond = g.precond;
        gc->gen = g_shape_gen.load();
    }
    if (gc->failed[kind]) {
        chunk_direct<T>(kind, g);
        return;
    }
    if (!gc->exec[kind]) {
        cudaGraph_t graph = nullptr;
        int nk = 0;
        cudaError_t e = cudaSuccess;
        t_capturing = true;
        if (kind == 1 && g_cond_nodes) {
            e = capture_pf_chunk<T>(g, &graph, &nk);
        } else {
            e = cudaStreamBeginCapture(g.st, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                chunk_direct<T>(kind, g);
                e = cudaStreamEndCapture(g.st, &graph);
            }
            if (graph) {
                size_t n = 0;
                cudaGraphGetNodes(graph, nullptr, &n);
                nk = (int)n;
            }
        }
        t_capturing = false;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&gc->exec[kind], graph, 0);
        if (graph) {
            gc->nodes[kind] = nk;
            cudaGraphDestroy(graph);
        }
        if (e != cudaSuccess) {
            take_launch_error();   // the capture failed; the chunk is launched directly instead
            gc->exec[kind] = nullptr;
            gc->failed[kind] = true;
            chunk_direct<T>(kind, g);
            return;
        }
    }
    cudaGraphLaunch(gc->exec[kind], g.st);
    g_launches.fetch_add((unsigned long long)gc->nodes[kind], std::memory_order_relaxed);
}

template <typename T>
static int poll(Group& g, bool ctrl_too, pff_problem* eh) {
    const Desc<T>* d = (const Desc<T>*)g.d_desc;
    cudaError_t e = take_launch_error();
    if (e != cudaSuccess) return cuda_fail(eh, e, "kernel launch");
    launch_gather<T>(d, g.np, g.d_flags, ctrl_too ? (void*)g.d_ctrl : nullptr, g.st);
    e = cudaMemcpyAsync(g.h_flags, g.d_flags, sizeof(int) * g.np, cudaMemcpyDeviceToHost, g.st);
    if (e == cudaSuccess && ctrl_too)
        e = cudaMemcpyAsync(g.h_ctrl, g.d_ctrl, sizeof(Ctrl) * g.np, cudaMemcpyDeviceToHost, g.st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g.st);
    if (e != cudaSuccess) return cuda_fail(eh, e, "poll");
    if (timing_on()) timing_collect();
    return 0;
}

static bool all_bits(const Group& g, int bit) {
    for (int j = 0; j < g.np; ++j)
        if (!(g.h_flags[j] & bit)) return false;
    return true;
}

// Mechanics sub-problem (Newton rounds of CG solves) for every problem of g.
template <typename T>
static int mech_solve_group(Group& g, int max_cg, int max_newton, pff_problem* eh, bool& warmed) {
    const Desc<T>* d = (const Desc<T>*)g.d_desc;
    const int nx = g.nx, ny = g.ny, wp = g.wp, np = g.np;
    cudaStream_t st = g.st;
    int rc;
    if (mech_cluster_group<T>(g)) return 0;
    for (int round = 0; round <= max_newton; ++round) {
        launch_row_fwd<T>(RF_NEWTON, nx, ny, d, np, st);
        launch_col<T>(CO_GAMMA_N, nx, ny, wp, d, np, st);
        launch_row_inv<T>(RI_NEWTON, nx, ny, d, np, st);
        for (int it = 0; it <= max_cg + CHUNK; it += CHUNK) {
            run_chunk<T>(0, g, warmed);
            if ((rc = poll<T>(g, false, eh))) return rc;
            if (all_bits(g, 1)) break;
        }
        if (all_bits(g, 2)) break;
    }
    launch_elem<T>(EL_FOLD, nx, ny, d, np, st);
    return 0;
}

// lap = nabla^2_N phi; with_df: the driving-force maximum and rescale of Algorithm 4.
template <typename T>
static void lap_phi_group(Group& g, bool with_df) {
    const Desc<T>* d = (const Desc<T>*)g.d_desc;
    launch_row_fwd<T>(RF_PHI, g.nx, g.ny, d, g.np, g.st);
    launch_col<T>(CO_LAP_DF, g.nx, g.ny, g.wp, d, g.np, g.st);
    launch_row_inv<T>(RI_LAP, g.nx, g.ny, d, g.np, g.st);
    if (with_df) launch_elem<T>(EL_DF, g.nx, g.ny, d, g.np, g.st);
}

// Phase-field sub-problem (Algorithm 1) followed by the post-step kernel.  A
// single FP32 512 x 512 problem runs the whole solve in one persistent
// cooperative launch (k_persist.cu) when enabled; otherwise chunks of CHUNK
// iterations are launched (graph replays) and polled.
template <typename T>
static int pf_solve_group(Group& g, int max_pf, pff_problem* eh, bool& warmed) {
    const Desc<T>* d = (const Desc<T>*)g.d_desc;
    int rc;
    launch_elem<T>(EL_PF_INIT, g.nx, g.ny, d, g.np, g.st);
    if constexpr (sizeof(T) == 4) {
        if (g_persist && !g.precond && g.np == 1 && g.nx == 512 && g.ny == 512 && !timing_on()) {
            cudaError_t e = launch_persist_bccg((const Desc<float>*)g.d_desc, max_pf + 2,
                                                persist_bccg_blocks(g_persist_share), g.st);
            if (e == cudaSuccess) {
                if ((rc = poll<T>(g, true, eh))) return rc;
                if (g.h_ctrl[0].status & 8)
                    return fail(eh, PFF_ERR_BARRIER_TIMEOUT, "persistent phase-field solve: a grid barrier timed out");
                launch_elem<T>(EL_POST, g.nx, g.ny, d, g.np, g.st);
                return 0;
            }
            cudaGetLastError();   // not launched (e.g. not enough resident capacity): chunked path
        }
    }
    for (int it = 0; it <= max_pf + CHUNK; it += CHUNK) {
        run_chunk<T>(1, g, warmed);
        if ((rc = poll<T>(g, false, eh))) return rc;
        if (all_bits(g, 4)) break;
    }
    launch_elem<T>(EL_POST, g.nx, g.ny, d, g.np, g.st);
    return 0;
}

// One load step (one pass of Algorithm 4's loop) for every problem of g.
template <typename T>
static int step_group(Group& g, int max_cg, int max_pf, int max_newton, bool energies, pff_problem* eh) {
    const Desc<T>* d = (const Desc<T>*)g.d_desc;
    int rc;
    bool warmed = g.graphs && (g.graphs->exec[0] || g.graphs->exec[1]);
    launch_step_begin<T>(d, g.np, g.st);
    if ((rc = mech_solve_group<T>(g, max_cg, max_newton, eh, warmed))) return rc;
    lap_phi_group<T>(g, true);                      // Algorithm 4 lines 4-10
    if ((rc = pf_solve_group<T>(g, max_pf, eh, warmed))) return rc;   // lines 11-14
    if (energies) {
        launch_row_fwd<T>(RF_PHI, g.nx, g.ny, d, g.np, g.st);
        launch_col<T>(CO_LAP_PLAIN, g.nx, g.ny, g.wp, d, g.np, g.st);
        launch_row_inv<T>(RI_ENERGY, g.nx, g.ny, d, g.np, g.st);
    }
    cudaError_t e = take_launch_error();
    if (e != cudaSuccess) return cuda_fail(eh, e, "kernel launch");
    return poll<T>(g, true, eh);
}

static void fill_report(const Ctrl& c, int split, pff_step_report* r) {
    for (int j = 0; j < 3; ++j) { r->eps_bar[j] = c.rep_eps_bar[j]; r->sig_bar[j] = c.sig_bar[j]; }
    r->C_bar = c.C_bar;
    r->gamma = c.gamma;
    r->dphi_L1 = c.dphi;
    r->F_e = c.Fe;
    r->F_f = c.Ff;
    r->mF_max = c.mF_max;
    r->D_max = c.D_max;
    r->mech_res = (contact_of(split) == ISOTROPIC && c.newton_it > 0) ? std::sqrt(c.rr) : std::sqrt(c.R2);
    r->pf_res = std::sqrt(c.pf_rr);
    r->rescaled = c.rescaled;
    r->incremented = c.incremented;
    r->newton_iters = c.newton_it;
    r->mech_cg_iters = c.cg_total;
    r->bccg_iters = c.pf_it;
    r->n_active = c.n_active;
    r->bccg_clamp_iters = c.pf_clamp_iters;
    r->bccg_full_iters = c.pf_full_iters;
    r->dt = 0.0;
    r->inner_iters = 0;
    r->istar = c.istar;
    r->broken = c.broken;
    r->status = (c.status & 8) ? PFF_ERR_BARRIER_TIMEOUT : c.status ? PFF_ERR_NOT_CONVERGED : PFF_OK;
}

static Group single_group(pff_problem* h) {
    Group g;
    g.nx = h->nx; g.ny = h->ny; g.wp = h->wp; g.prec = h->prec; g.np = 1;
    g.st = h->st;
    g.d_desc = h->d_desc;
    g.d_flags = h->d_flags;
    g.d_ctrl = h->d_ctrlcopy;
    g.h_flags = h->h_flags;
    g.h_ctrl = h->h_ctrl;
    g.graphs = &h->graphs;
    g.precond = h->prm.pf_precondition != 0;
    return g;
}

static int run_group_step(Group& g, const pff_params& p, bool energies, pff_problem* eh) {
    if (g.prec == PFF_FP64)
        return step_group<double>(g, p.mech_max_cg, p.pf_max_iter, p.mech_max_newton, energies, eh);
    return step_group<float>(g, p.mech_max_cg, p.pf_max_iter, p.mech_max_newton, energies, eh);
}

template <typename T>
static void run_trio(pff_problem* h, int rf, int co, int ri) {
    const Desc<T>* d = (const Desc<T>*)h->d_desc;
    launch_row_fwd<T>(rf, h->nx, h->ny, d, 1, h->st);
    launch_col<T>(co, h->nx, h->ny, h->wp, d, 1, h->st);
    launch_row_inv<T>(ri, h->nx, h->ny, d, 1, h->st);
}
static void trio(pff_problem* h, int rf, int co, int ri) {
    if (h->prec == PFF_FP64) run_trio<double>(h, rf, co, ri);
    else run_trio<float>(h, rf, co, ri);
}
static void elem(pff_problem* h, int op) {
    if (h->prec == PFF_FP64) launch_elem<double>(op, h->nx, h->ny, (const Desc<double>*)h->d_desc, 1, h->st);
    else launch_elem<float>(op, h->nx, h->ny, (const Desc<float>*)h->d_desc, 1, h->st);
}
static int sync(pff_problem* h, const char* where) {
    cudaError_t e = take_launch_error();
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    return e == cudaSuccess ? 0 : cuda_fail(h, e, where);
}


// ---------------------------------------------------------------------------- Algorithms 2 and 3
static int set_method_ctrl(pff_problem* h, int use_override, double eta_dt, int frozen, int post_mode) {
    int rc = read_ctrl(h);
    if (rc) return rc;
    h->h_ctrl->use_override = use_override;
    h->h_ctrl->eta_dt_override = eta_dt;
    h->h_ctrl->con_frozen = frozen;
    h->h_ctrl->post_mode = post_mode;
    return write_ctrl(h);
}

static int add_increment(pff_problem* h) {
    int rc = read_ctrl(h);
    if (rc) return rc;
    for (int j = 0; j < 3; ++j) h->h_ctrl->eps_bar[j] += h->prm.d_eps_bar[j];
    return write_ctrl(h);
}

// One strain increment of Algorithm 2: eps_bar += d_eps_bar, then alternating
// mechanics / phase-field solves (eta/dt = 0, phi_con of the increment's start)
// until ||phi_{s,n+1} - phi_{s,n}||_1 < Tol_AM.
template <typename T>
static int am_increment(pff_problem* h, pff_step_report* out) {
    Group g = single_group(h);
    const pff_params& p = h->prm;
    const Desc<T>* d = (const Desc<T>*)h->d_desc;
    int rc;
    if ((rc = add_increment(h))) return rc;
    launch_elem<T>(EL_SAVE_CON, h->nx, h->ny, d, 1, h->st);
    if ((rc = set_method_ctrl(h, 1, 0.0, 1, 1))) return rc;
    bool warmed = h->graphs.exec[0] || h->graphs.exec[1];
    int inner = 0, cg = 0, pf = 0, clamps = 0, fulls = 0, status = 0;
    double dphi = 0.0;
    do {
        launch_step_begin<T>(d, 1, h->st);
        if ((rc = mech_solve_group<T>(g, p.mech_max_cg, p.mech_max_newton, h, warmed))) break;
        lap_phi_group<T>(g, false);
        if ((rc = pf_solve_group<T>(g, p.pf_max_iter, h, warmed))) break;
        if ((rc = poll<T>(g, true, h))) break;
        const Ctrl& c = g.h_ctrl[0];
        dphi = c.dphi;
        cg += c.cg_total;
        pf += c.pf_it;
        clamps += c.pf_clamp_iters;
        fulls += c.pf_full_iters;
        status |= c.status;
        ++inner;
    } while (dphi >= p.tol_am && inner < p.am_max_inner);
    int rc2 = set_method_ctrl(h, 0, 0.0, 0, 0);
    if (rc) return rc;
    if (rc2) return rc2;
    if (out) {
        fill_report(g.h_ctrl[0], h->split, out);
        out->mech_cg_iters = cg;
        out->bccg_iters = pf;
        out->bccg_clamp_iters = clamps;
        out->bccg_full_iters = fulls;
        out->inner_iters = inner;
        out->incremented = 1;
        out->status = status || inner >= p.am_max_inner ? PFF_ERR_NOT_CONVERGED : PFF_OK;
    }
    return PFF_OK;
}

// One time step of Algorithm 3: mechanics at (eps_bar_n, phi_n), then phase-field
// solves with dt halved until ||dphi||_1 < (dphi)_max or dt <= (dt)_min (dt doubled,
// up to (dt)_max, after an easy step); eps_bar grows when ||dphi||_1 < (dphi)_min at dt >= (dt)_max.
template <typename T>
static int td_step(pff_problem* h, pff_step_report* out) {
    Group g = single_group(h);
    const pff_params& p = h->prm;
    const Desc<T>* d = (const Desc<T>*)h->d_desc;
    int rc;
    if (h->td_dt <= 0.0) h->td_dt = p.dt_max;
    double dt = h->td_dt;
    bool warmed = h->graphs.exec[0] || h->graphs.exec[1];
    if ((rc = set_method_ctrl(h, 1, p.Gc / p.ell / dt, 0, 1))) return rc;
    launch_step_begin<T>(d, 1, h->st);
    if ((rc = mech_solve_group<T>(g, p.mech_max_cg, p.mech_max_newton, h, warmed))) return rc;
    lap_phi_group<T>(g, false);
    launch_elem<T>(EL_SAVE_PHI, h->nx, h->ny, d, 1, h->st);
    int tries = 0, pf = 0, clamps = 0, fulls = 0, status = 0;
    double dphi = 0.0;
    for (;;) {
        if (tries > 0 && (rc = set_method_ctrl(h, 1, p.Gc / p.ell / dt, 0, 1))) return rc;
        if ((rc = pf_solve_group<T>(g, p.pf_max_iter, h, warmed))) return rc;
        if ((rc = poll<T>(g, true, h))) return rc;
        const Ctrl& c = g.h_ctrl[0];
        dphi = c.dphi;
        pf += c.pf_it;
        clamps += c.pf_clamp_iters;
        fulls += c.pf_full_iters;
        status |= c.status;
        ++tries;
        if (dphi < p.dphi_max || dt <= p.dt_min || tries >= 64) {
            if (dphi < 0.5 * p.dphi_max) dt = std::min(2.0 * dt, p.dt_max);
            break;
        }
        dt *= 0.5;
        launch_elem<T>(EL_RESTORE_PHI, h->nx, h->ny, d, 1, h->st);   // retry from phi_n
        lap_phi_group<T>(g, false);   // the solve's initial residual overwrote nabla^2 phi_n
    }
    Ctrl c = g.h_ctrl[0];
    h->td_dt = dt;
    bool inc = dphi < p.dphi_min && dt >= p.dt_max;
    if ((rc = set_method_ctrl(h, 0, 0.0, 0, 0))) return rc;
    if (inc && (rc = add_increment(h))) return rc;
    if (out) {
        fill_report(c, h->split, out);
        out->bccg_iters = pf;
        out->bccg_clamp_iters = clamps;
        out->bccg_full_iters = fulls;
        out->inner_iters = tries;
        out->incremented = inc;
        out->dt = dt;
        out->status = status ? PFF_ERR_NOT_CONVERGED : PFF_OK;
    }
    return PFF_OK;
}

// ---------------------------------------------------------------------------- batching
struct BatchGroup {
    int nx = 0, ny = 0, prec = 0, precond = 0;
    std::vector<int> slots;
    int cap = 0;
    void* d_desc = nullptr;
    int* d_flags = nullptr;
    Ctrl* d_ctrl = nullptr;
    int* h_flags = nullptr;
    Ctrl* h_ctrl = nullptr;
    GraphCache* graphs = nullptr;
    cudaStream_t stream = nullptr;   // own stream: groups of different shapes overlap on the device
};

}  // namespace pff

struct pff_batch {
    int max_slots = 0;
    int group_cap = 0;            // max problems per launch group (0: all of a shape)
    size_t budget = 0, used = 0;
    cudaStream_t st = nullptr;
    std::vector<pff_problem*> slot;
    std::vector<pff::BatchGroup> groups;
    std::string err;
};

namespace pff {

static void free_group(BatchGroup& g) {
    if (g.stream) { cudaStreamSynchronize(g.stream); cudaStreamDestroy(g.stream); }
    if (g.graphs) { g.graphs->reset(); delete g.graphs; }
    if (g.d_desc) cudaFree(g.d_desc);
    if (g.d_flags) cudaFree(g.d_flags);
    if (g.d_ctrl) cudaFree(g.d_ctrl);
    if (g.h_flags) cudaFreeHost(g.h_flags);
    if (g.h_ctrl) cudaFreeHost(g.h_ctrl);
    g = BatchGroup();
}

// (Re)build the groups of live problems: equal (nx, ny, precision) share launches.
static int build_groups(pff_batch* b) {
    std::map<std::tuple<int, int, int, int>, std::vector<int>> by;
    for (int i = 0; i < b->max_slots; ++i) {
        pff_problem* h = b->slot[i];
        if (h && !h->broken) by[std::make_tuple(h->nx, h->ny, h->prec, h->prm.pf_precondition != 0)].push_back(i);
    }
    // split each shape into launch groups of at most group_cap problems
    std::vector<std::pair<std::tuple<int, int, int, int>, std::vector<int>>> parts;
    for (auto& kv : by) {
        const int cap = b->group_cap > 0 ? b->group_cap : (int)kv.second.size();
        for (size_t i0 = 0; i0 < kv.second.size(); i0 += cap)
            parts.emplace_back(kv.first, std::vector<int>(kv.second.begin() + i0,
                                                          kv.second.begin() + std::min(kv.second.size(), i0 + cap)));
    }
    std::vector<BatchGroup> next;
    for (auto& kv : parts) {
        BatchGroup g;
        g.nx = std::get<0>(kv.first);
        g.ny = std::get<1>(kv.first);
        g.prec = std::get<2>(kv.first);
        g.precond = std::get<3>(kv.first);
        g.slots = kv.second;
        // reuse buffers of an old group of the same shape when large enough
        for (auto& old : b->groups)
            if (old.d_desc && old.nx == g.nx && old.ny == g.ny && old.prec == g.prec && old.precond == g.precond &&
                old.cap >= (int)g.slots.size()) {
                g.cap = old.cap; g.d_desc = old.d_desc; g.d_flags = old.d_flags; g.d_ctrl = old.d_ctrl;
                g.h_flags = old.h_flags; g.h_ctrl = old.h_ctrl; g.graphs = old.graphs; g.stream = old.stream;
                old.d_desc = nullptr; old.d_flags = nullptr; old.d_ctrl = nullptr; old.h_flags = nullptr; old.h_ctrl = nullptr;
                old.graphs = nullptr; old.stream = nullptr;
                break;
            }
        if (!g.d_desc) {
            g.cap = (int)g.slots.size();
            cudaError_t e = cudaMalloc(&g.d_desc, sizeof(Desc<double>) * g.cap);
            if (e == cudaSuccess) e = cudaMalloc((void**)&g.d_flags, sizeof(int) * g.cap);
            if (e == cudaSuccess) e = cudaMalloc((void**)&g.d_ctrl, sizeof(Ctrl) * g.cap);
            if (e == cudaSuccess) e = cudaMallocHost((void**)&g.h_flags, sizeof(int) * g.cap);
            if (e == cudaSuccess) e = cudaMallocHost((void**)&g.h_ctrl, sizeof(Ctrl) * g.cap);
            if (e != cudaSuccess) { free_group(g); b->err = cudaGetErrorString(e); return PFF_ERR_CUDA; }
        }
        if (!g.graphs) g.graphs = new GraphCache();
        if (!g.stream && parts.size() > 1) {
            if (cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking) != cudaSuccess) {
                cudaGetLastError();
                g.stream = nullptr;
            }
        }
        next.push_back(g);
    }
    for (auto& old : b->groups) free_group(old);
    b->groups = next;
    // descriptors (parameters may have changed since the last step)
    for (auto& g : b->groups) {
        std::vector<Desc<double>> hd(g.slots.size());
        for (size_t j = 0; j < g.slots.size(); ++j) {
            pff_problem* h = b->slot[g.slots[j]];
            if (g.prec == PFF_FP64) hd[j] = make_desc<double>(h);
            else { Desc<float> f = make_desc<float>(h); std::memcpy(&hd[j], &f, sizeof(f)); }
        }
        cudaError_t e = cudaMemcpyAsync(g.d_desc, hd.data(), sizeof(Desc<double>) * hd.size(), cudaMemcpyHostToDevice, b->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
        if (e != cudaSuccess) { b->err = cudaGetErrorString(e); return PFF_ERR_CUDA; }
    }
    return PFF_OK;
}

}  // namespace pff

// ============================================================================ C ABI
extern "C" {

int pff_default_params(pff_params* p) {
    if (!p) return PFF_ERR_INVALID_ARG;
    std::memset(p, 0, sizeof(*p));
    p->nu = 0.2;
    p->Gc = 1.0;
    p->ell = 1.0;
    p->dx = 1.0;
    p->mech_tol = 1e-6;
    p->mech_cg_rtol = 1e-4;
    p->mech_max_newton = 50;
    p->mech_max_cg = 5000;
    p->pf_tol = 1e-6;
    p->pf_atol = 1e-12;
    p->pf_max_iter = 20000;
    p->eta_over_dt = -1.0;
    p->F_max = -1.0;
    p->thresh = -1.0;
    p->dphi_min = 1e-3;
    p->C_broken = -1.0;
    p->crack_set_threshold = 0.9;
    p->d_eps_bar[0] = 0.0;
    p->d_eps_bar[1] = 1e-4;
    p->d_eps_bar[2] = 0.0;
    p->compute_energies = 1;
    p->evolution = PFF_NEAR_EQUILIBRIUM;
    p->tol_am = 1e-3;
    p->am_max_inner = 1000;
    p->dt_min = std::ldexp(1.0, -16);
    p->dt_max = std::ldexp(1.0, 16);
    p->dphi_max = 1.5;
    p->pf_precondition = 0;
    return PFF_OK;
}

size_t pff_problem_bytes(int nx, int ny, int precision) { return problem_bytes(nx, ny, precision); }

int pff_create_problem(int nx, int ny, int precision, void* cuda_stream, pff_problem** out) {
    if (!out) return PFF_ERR_INVALID_ARG;
    *out = nullptr;
    if (!valid_n(nx) || !valid_n(ny) || (precision != PFF_FP64 && precision != PFF_MIXED)) return PFF_ERR_INVALID_ARG;
    pff_problem* h = new pff_problem();
    h->nx = nx;
    h->ny = ny;
    h->prec = precision;
    h->wp = wp_of(nx);
    h->st = (cudaStream_t)cuda_stream;
    cudaGetDevice(&h->dev);
    pff_default_params(&h->prm);
    if (twiddles_for(h->dev, h->tw)) { delete h; return PFF_ERR_CUDA; }
    const size_t n = h->n();
    const size_t es = precision == PFF_FP64 ? 8 : 4;
    h->bytes = problem_bytes(nx, ny, precision);
    cudaError_t e = cudaMalloc((void**)&h->base, h->bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return e == cudaErrorMemoryAllocation ? PFF_ERR_OOM : PFF_ERR_CUDA;
    }
    char* p = h->base;
    for (int f = 0; f < NFIELDS; ++f) { h->field[f] = p; p += align256(n * es); }
    h->flags = (uint8_t*)p; p += align256(n);
    h->S = p; p += align256((size_t)3 * ny * h->wp * 2 * es);
    h->part = (double*)p; p += align256((size_t)PART_BLOCKS * 8 * sizeof(double));
    if (precision != PFF_FP64) { h->stage = (double*)p; p += align256(n * sizeof(double)); }
    h->ctrl = (Ctrl*)p;
    e = cudaMemsetAsync(h->base, 0, h->bytes, h->st);
    if (e == cudaSuccess) e = cudaMalloc(&h->d_desc, sizeof(Desc<double>));
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->d_flags, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->d_ctrlcopy, sizeof(Ctrl));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&h->h_flags, sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&h->h_ctrl, sizeof(Ctrl));
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) {
        pff_destroy_problem(h);
        return PFF_ERR_CUDA;
    }
    // E = 1 everywhere
    std::vector<double> ones(n, 1.0);
    if (pff_set_modulus_field(h, ones.data(), 0)) { pff_destroy_problem(h); return PFF_ERR_CUDA; }
    *out = h;
    return PFF_OK;
}

int pff_destroy_problem(pff_problem* h) {
    if (!h) return PFF_ERR_INVALID_ARG;
    if (h->st) cudaStreamSynchronize(h->st);
    else cudaDeviceSynchronize();
    if (h->base) cudaFree(h->base);
    if (h->d_desc) cudaFree(h->d_desc);
    if (h->d_flags) cudaFree(h->d_flags);
    if (h->d_ctrlcopy) cudaFree(h->d_ctrlcopy);
    if (h->h_flags) cudaFreeHost(h->h_flags);
    if (h->h_ctrl) cudaFreeHost(h->h_ctrl);
    h->graphs.reset();
    delete h;
    return PFF_OK;
}

const char* pff_last_error(pff_problem* h) { return h ? h->err.c_str() : "null handle"; }

int pff_problem_info(pff_problem* h, int* nx, int* ny, int* precision) {
    if (!h) return PFF_ERR_INVALID_ARG;
    if (nx) *nx = h->nx;
    if (ny) *ny = h->ny;
    if (precision) *precision = h->prec;
    return PFF_OK;
}

int pff_set_params(pff_problem* h, const pff_params* p) {
    if (!h || !p) return PFF_ERR_INVALID_ARG;
    if (!(p->nu > -1.0 && p->nu < 0.5) || !(p->Gc > 0) || !(p->ell > 0) || !(p->dx > 0) || p->mech_max_cg < 1 ||
        p->pf_max_iter < 1 || p->mech_max_newton < 1 || p->evolution < PFF_NEAR_EQUILIBRIUM ||
        p->evolution > PFF_TIME_DEPENDENT || !(p->dt_min > 0) || !(p->dt_max >= p->dt_min) || p->am_max_inner < 1)
        return fail(h, PFF_ERR_INVALID_ARG, "invalid parameter value");
    h->prm = *p;
    return upload_desc(h);
}

int pff_get_params(pff_problem* h, pff_params* p) {
    if (!h || !p) return PFF_ERR_INVALID_ARG;
    *p = h->prm;
    return PFF_OK;
}

int pff_set_model(pff_problem* h, int fracture, int split, int irreversibility) {
    if (!h) return PFF_ERR_INVALID_ARG;
    if ((fracture != PFF_AT1 && fracture != PFF_AT2) ||
        (split < PFF_ISOTROPIC || split > PFF_SPECTRAL_VOLDEV) ||
        (irreversibility != PFF_CRACK_SET && irreversibility != PFF_DAMAGE))
        return fail(h, PFF_ERR_INVALID_ARG, "invalid model selector");
    h->fracture = fracture;
    h->split = split;
    h->irrev = irreversibility;
    return upload_desc(h);
}

int pff_set_modulus_field(pff_problem* h, const double* E, int on_device) {
    if (!h || !E) return PFF_ERR_INVALID_ARG;
    const size_t n = h->n();
    double s = 0.0, s2 = 0.0;
    if (on_device) {
        std::vector<double> tmp(n);
        cudaError_t e = cudaMemcpyAsync(tmp.data(), E, n * 8, cudaMemcpyDeviceToHost, h->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
        if (e != cudaSuccess) return cuda_fail(h, e, "read modulus");
        for (size_t i = 0; i < n; ++i) { s += tmp[i]; s2 += tmp[i] * tmp[i]; }
        for (size_t i = 0; i < n; ++i)
            if (!(tmp[i] >= 0.0) || !std::isfinite(tmp[i])) return fail(h, PFF_ERR_INVALID_ARG, "E must be non-negative and finite");
    } else {
        for (size_t i = 0; i < n; ++i) {
            if (!(E[i] >= 0.0) || !std::isfinite(E[i])) return fail(h, PFF_ERR_INVALID_ARG, "E must be non-negative and finite");
            s += E[i];
            s2 += E[i] * E[i];
        }
    }
    if (!(s > 0.0)) return fail(h, PFF_ERR_INVALID_ARG, "E must have a positive mean");
    int rc = put_field(h, h->field[0], E, n, on_device);
    if (rc) return rc;
    if (s == h->sumE && s2 == h->sumE2) return PFF_OK;   // the same sums: control block and constants unchanged
    h->sumE = s;
    h->sumE2 = s2;
    // the two sums only (adjacent in the control block), from the pinned host mirror
    static_assert(offsetof(Ctrl, sumE) == offsetof(Ctrl, sumE2) + sizeof(double), "sumE2, sumE adjacent");
    h->h_ctrl->sumE2 = s2;
    h->h_ctrl->sumE = s;
    cudaError_t e = cudaMemcpyAsync(&h->ctrl->sumE2, &h->h_ctrl->sumE2, 2 * sizeof(double), cudaMemcpyHostToDevice, h->st);
    if (e != cudaSuccess) return cuda_fail(h, e, "write modulus sums");
    return upload_desc(h);   // C_broken follows the mean modulus; synchronises the stream
}

int pff_init_crack(pff_problem* h, int target, int shape, double xc, double yc, double length, double E0) {
    if (!h) return PFF_ERR_INVALID_ARG;
    if (target != PFF_IC_PHASE_FIELD && target != PFF_IC_MODULUS)
        return fail(h, PFF_ERR_INVALID_ARG, "target must be PFF_IC_PHASE_FIELD or PFF_IC_MODULUS");
    if (shape != PFF_CRACK_SEGMENT && shape != PFF_CRACK_EDGE)
        return fail(h, PFF_ERR_INVALID_ARG, "shape must be PFF_CRACK_SEGMENT or PFF_CRACK_EDGE");
    if (!(length >= 0.0) || !std::isfinite(xc) || !std::isfinite(yc) || (target == PFF_IC_MODULUS && !(E0 > 0.0)))
        return fail(h, PFF_ERR_INVALID_ARG, "length must be >= 0, the centre finite and E0 > 0");
    const size_t n = h->n();
    double* buf = nullptr;
    cudaError_t e = cudaMalloc(&buf, n * 8);
    if (e != cudaSuccess) { cudaGetLastError(); return fail(h, PFF_ERR_OOM, "crack initial condition scratch"); }
    micro_crack(buf, h->nx, h->ny, h->prm.dx, h->prm.ell, xc, yc, length, shape, target == PFF_IC_MODULUS, E0, h->st);
    e = cudaGetLastError();
    int rc = e == cudaSuccess ? PFF_OK : cuda_fail(h, e, "crack initial condition");
    if (!rc) rc = target == PFF_IC_MODULUS ? pff_set_modulus_field(h, buf, 1) : pff_set_phase_field(h, buf, 1);
    cudaStreamSynchronize(h->st);
    cudaFree(buf);
    return rc;
}

int pff_default_micro_params(pff_micro_params* mp) {
    if (!mp) return PFF_ERR_INVALID_ARG;
    mp->kind = PFF_MICRO_RANDOM;
    mp->L_cut = 6.0;
    mp->std_target = 0.3;
    mp->xi_min = 0.01;
    mp->a = 0.875;
    mp->ac_iters = 21;
    mp->E0 = 1.0;
    return PFF_OK;
}

int pff_generate_modulus(pff_problem* h, const pff_micro_params* mp, const double* noise, int noise_on_device) {
    if (!h || !mp || !noise) return PFF_ERR_INVALID_ARG;
    if ((mp->kind != PFF_MICRO_RANDOM && mp->kind != PFF_MICRO_TWO_PHASE) || !(mp->L_cut > 0.0) || !(mp->E0 > 0.0) ||
        (mp->kind == PFF_MICRO_RANDOM && (!(mp->std_target > 0.0) || !(mp->xi_min < 1.0))) ||
        (mp->kind == PFF_MICRO_TWO_PHASE && (!(mp->a > 0.0) || !(mp->a < 1.0) || mp->ac_iters < 0)))
        return fail(h, PFF_ERR_INVALID_ARG, "invalid microstructure parameters");
    const size_t n = h->n();
    double *xi = nullptr, *E = nullptr;
    cudaError_t e = cudaMalloc(&xi, n * 8);
    if (e == cudaSuccess) e = cudaMalloc(&E, n * 8);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(xi);
        return fail(h, PFF_ERR_OOM, "microstructure scratch");
    }
    e = cudaMemcpyAsync(xi, noise, n * 8, noise_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->st);
    int rc = e == cudaSuccess ? PFF_OK : cuda_fail(h, e, "noise upload");
    std::string err;
    if (!rc) {
        rc = micro_generate(h->nx, h->ny, h->prm.dx, *mp, xi, E, h->tw.t64, h->st, err);
        if (rc) fail(h, rc, err);
    }
    if (!rc) rc = pff_set_modulus_field(h, E, 1);
    cudaStreamSynchronize(h->st);
    cudaFree(xi);
    cudaFree(E);
    return rc;
}

int pff_set_phase_field(pff_problem* h, const double* phi, int on_device) {
    if (!h || !phi) return PFF_ERR_INVALID_ARG;
    h->broken = false;
    return put_field(h, h->field[1], phi, h->n(), on_device);
}

int pff_set_strain(pff_problem* h, const double* eps_star, const double eps_bar[3], int on_device) {
    if (!h || !eps_bar) return PFF_ERR_INVALID_ARG;
    const size_t n = h->n();
    const size_t es = h->prec == PFF_FP64 ? 8 : 4;
    int rc;
    for (int j = 0; j < 3; ++j) {
        if (eps_star) {
            if ((rc = put_field(h, h->field[2 + j], eps_star + j * n, n, on_device))) return rc;
        } else {
            cudaError_t e = cudaMemsetAsync(h->field[2 + j], 0, n * es, h->st);
            if (e != cudaSuccess) return cuda_fail(h, e, "memset");
        }
    }
    if ((rc = read_ctrl(h))) return rc;
    for (int j = 0; j < 3; ++j) h->h_ctrl->eps_bar[j] = eps_bar[j];
    h->broken = false;
    h->td_dt = -1.0;
    return write_ctrl(h);
}

int pff_set_flag(pff_problem* h, int flag) {
    if (!h) return PFF_ERR_INVALID_ARG;
    int rc = read_ctrl(h);
    if (rc) return rc;
    h->h_ctrl->flag = flag ? 1 : 0;
    return write_ctrl(h);
}

int pff_step_load(pff_problem* h, int n_steps, pff_step_report* out, int* steps_done) {
    if (!h || n_steps < 0) return PFF_ERR_INVALID_ARG;
    if (steps_done) *steps_done = 0;
    Group g = single_group(h);
    int status = PFF_OK;
    if (h->prm.evolution != PFF_NEAR_EQUILIBRIUM) {
        for (int s = 0; s < n_steps; ++s) {
            pff_step_report rep;
            std::memset(&rep, 0, sizeof(rep));
            int rc;
            if (h->prm.evolution == PFF_ALTERNATING_MIN)
                rc = h->prec == PFF_FP64 ? am_increment<double>(h, &rep) : am_increment<float>(h, &rep);
            else
                rc = h->prec == PFF_FP64 ? td_step<double>(h, &rep) : td_step<float>(h, &rep);
            if (rc) return rc;
            if (out) out[s] = rep;
            if (rep.status) status = PFF_ERR_NOT_CONVERGED;
            if (steps_done) *steps_done = s + 1;
            if (rep.broken) { h->broken = true; break; }
        }
        if (status) h->err = "a sub-solver reached its iteration cap";
        return status;
    }
    for (int s = 0; s < n_steps; ++s) {
        int rc = run_group_step(g, h->prm, h->prm.compute_energies != 0, h);
        if (rc) return rc;
        const Ctrl& c = g.h_ctrl[0];
        if (out) fill_report(c, h->split, &out[s]);
        if (c.status) status = PFF_ERR_NOT_CONVERGED;
        if (steps_done) *steps_done = s + 1;
        if (c.broken) { h->broken = true; break; }
    }
    if (status) h->err = "a sub-solver reached its iteration cap";
    return status;
}

int pff_solve_mechanics(pff_problem* h, pff_step_report* out) {
    if (!h) return PFF_ERR_INVALID_ARG;
    Group g = single_group(h);
    const pff_params& p = h->prm;
    int rc;
    auto body = [&](auto tag) -> int {
        using T = decltype(tag);
        const Desc<T>* d = (const Desc<T>*)h->d_desc;
        launch_step_begin<T>(d, 1, h->st);
        if (mech_cluster_group<T>(g)) return poll<T>(g, true, h);
        for (int round = 0; round <= p.mech_max_newton; ++round) {
            run_trio<T>(h, RF_NEWTON, CO_GAMMA_N, RI_NEWTON);
            for (int it = 0; it <= p.mech_max_cg + CHUNK; it += CHUNK) {
                for (int c = 0; c < CHUNK; ++c) run_trio<T>(h, RF_CG, CO_GAMMA_CG, RI_CG);
                int r2 = poll<T>(g, false, h);
                if (r2) return r2;
                if (all_bits(g, 1)) break;
            }
            if (all_bits(g, 2)) break;
        }
        launch_elem<T>(EL_FOLD, h->nx, h->ny, d, 1, h->st);
        return poll<T>(g, true, h);
    };
    rc = h->prec == PFF_FP64 ? body(double()) : body(float());
    if (rc) return rc;
    if (out) {
        std::memset(out, 0, sizeof(*out));
        fill_report(g.h_ctrl[0], h->split, out);
    }
    return g.h_ctrl[0].status ? PFF_ERR_NOT_CONVERGED : PFF_OK;
}

int pff_solve_phase_field(pff_problem* h, pff_step_report* out) {
    if (!h) return PFF_ERR_INVALID_ARG;
    Group g = single_group(h);
    const pff_params& p = h->prm;
    // rescale disabled for a bare sub-problem: gamma = 1
    auto body = [&](auto tag) -> int {
        using T = decltype(tag);
        const Desc<T>* d = (const Desc<T>*)h->d_desc;
        launch_step_begin<T>(d, 1, h->st);
        run_trio<T>(h, RF_PHI, CO_LAP_PLAIN, RI_LAP);
        launch_elem<T>(EL_PF_INIT, h->nx, h->ny, d, 1, h->st);
        if constexpr (sizeof(T) == 4) {
            if (g_persist && !h->prm.pf_precondition && h->nx == 512 && h->ny == 512 && !timing_on()) {
                cudaError_t e = launch_persist_bccg((const Desc<float>*)h->d_desc, p.pf_max_iter + 2,
                                                    persist_bccg_blocks(1), h->st);
                if (e == cudaSuccess) {
                    int r2 = poll<T>(g, true, h);
                    if (r2) return r2;
                    if (g.h_ctrl[0].status & 8)
                        return fail(h, PFF_ERR_BARRIER_TIMEOUT, "persistent phase-field solve: a grid barrier timed out");
                    return 0;
                }
                cudaGetLastError();
            }
        }
        for (int it = 0; it <= p.pf_max_iter + CHUNK; it += CHUNK) {
            for (int c = 0; c < CHUNK; ++c) {
                if (p.pf_precondition || g_bccg4.load()) {
                    if (p.pf_precondition) run_trio<T>(h, RF_PF_Z, CO_PRECOND, RI_PF_Z);
                    run_trio<T>(h, RF_PF_A, CO_LAP_PF, RI_PF_A);
                    launch_elem<T>(EL_PF_B, h->nx, h->ny, d, 1, h->st);
                } else {
                    run_trio<T>(h, RF_PF_A, CO_LAP_PFQ, RI_PF_AB);
                }
                run_trio<T>(h, RF_PF_B, CO_LAP_PF_FULL, RI_PF_B);
            }
            int r2 = poll<T>(g, false, h);
            if (r2) return r2;
            if (all_bits(g, 4)) break;
        }
        // phi += v without touching eps_bar: only the update of FPost is wanted, so run
        // it and restore eps_bar afterwards
        return poll<T>(g, true, h);
    };
    int rc = h->prec == PFF_FP64 ? body(double()) : body(float());
    if (rc) return rc;
    Ctrl saved = g.h_ctrl[0];
    elem(h, EL_POST);
    if ((rc = sync(h, "phase-field update"))) return rc;
    if ((rc = read_ctrl(h))) return rc;
    for (int j = 0; j < 3; ++j) h->h_ctrl->eps_bar[j] = saved.eps_bar[j];
    Ctrl post = *h->h_ctrl;
    if ((rc = write_ctrl(h))) return rc;
    if (out) {
        std::memset(out, 0, sizeof(*out));
        fill_report(post, h->split, out);
        out->bccg_iters = saved.pf_it;
        out->pf_res = std::sqrt(saved.pf_rr);
        out->n_active = saved.n_active;
        out->incremented = 0;
        for (int j = 0; j < 3; ++j) out->eps_bar[j] = saved.eps_bar[j];
    }
    return saved.status ? PFF_ERR_NOT_CONVERGED : PFF_OK;
}

int pff_get_fields(pff_problem* h, int which, double* host_out) {
    if (!h || !host_out) return PFF_ERR_INVALID_ARG;
    const size_t n = h->n();
    int rc;
    switch (which) {
        case PFF_FIELD_EPS_STAR:
            for (int j = 0; j < 3; ++j)
                if ((rc = get_field(h, h->field[2 + j], host_out + j * n, n))) return rc;
            return PFF_OK;
        case PFF_FIELD_STRAIN: {
            if ((rc = read_ctrl(h))) return rc;
            double eb[3] = {h->h_ctrl->eps_bar[0], h->h_ctrl->eps_bar[1], h->h_ctrl->eps_bar[2]};
            for (int j = 0; j < 3; ++j) {
                if ((rc = get_field(h, h->field[2 + j], host_out + j * n, n))) return rc;
                for (size_t i = 0; i < n; ++i) host_out[j * n + i] += eb[j];
            }
            return PFF_OK;
        }
        case PFF_FIELD_PHI: return get_field(h, h->field[1], host_out, n);
        case PFF_FIELD_MODULUS: return get_field(h, h->field[0], host_out, n);
        case PFF_FIELD_UPDATE: return get_field(h, h->field[5], host_out, n);
        case PFF_FIELD_STRESS:
        case PFF_FIELD_PSI_PLUS: {
            elem(h, EL_STATE);
            if ((rc = sync(h, "state fields"))) return rc;
            if (which == PFF_FIELD_PSI_PLUS) return get_field(h, h->field[18], host_out, n);
            for (int j = 0; j < 3; ++j)
                if ((rc = get_field(h, h->field[14 + j], host_out + j * n, n))) return rc;
            return PFF_OK;
        }
        case PFF_FIELD_DRIVING_FORCE: {
            trio(h, RF_PHI, CO_LAP_PLAIN, RI_LAP);
            elem(h, EL_DRIVING);
            if ((rc = sync(h, "driving force"))) return rc;
            return get_field(h, h->field[11], host_out, n);
        }
        case PFF_FIELD_ACTIVE: {
            elem(h, EL_FLAGS);
            if ((rc = sync(h, "active set"))) return rc;
            return get_field(h, h->field[12], host_out, n);
        }
        default: return fail(h, PFF_ERR_INVALID_ARG, "unknown field selector");
    }
}

int pff_get_device_ptr(pff_problem* h, int which, void** p, int* dtype) {
    if (!h || !p) return PFF_ERR_INVALID_ARG;
    if (dtype) *dtype = h->prec == PFF_FP64 ? 0 : 1;
    switch (which) {
        case PFF_FIELD_EPS_STAR: *p = h->field[2]; return PFF_OK;
        case PFF_FIELD_PHI: *p = h->field[1]; return PFF_OK;
        case PFF_FIELD_MODULUS: *p = h->field[0]; return PFF_OK;
        default: return fail(h, PFF_ERR_INVALID_ARG, "field is not stored");
    }
}

int pff_apply_projection(pff_problem* h, const double* in3, double* out3) {
    if (!h || !in3 || !out3) return PFF_ERR_INVALID_ARG;
    const size_t n = h->n();
    int rc;
    for (int j = 0; j < 3; ++j)
        if ((rc = put_field(h, h->field[8 + j], in3 + j * n, n, 0))) return rc;
    trio(h, RF_COPY3, CO_GAMMA_PLAIN, RI_COPY3);
    if ((rc = sync(h, "projection"))) return rc;
    for (int j = 0; j < 3; ++j)
        if ((rc = get_field(h, h->field[14 + j], out3 + j * n, n))) return rc;
    return PFF_OK;
}

int pff_apply_laplacian(pff_problem* h, const double* in, double* out) {
    if (!h || !in || !out) return PFF_ERR_INVALID_ARG;
    const size_t n = h->n();
    int rc;
    if ((rc = put_field(h, h->field[8], in, n, 0))) return rc;
    trio(h, RF_COPY1, CO_LAP_PLAIN, RI_COPY1);
    if ((rc = sync(h, "laplacian"))) return rc;
    return get_field(h, h->field[14], out, n);
}

int pff_constitutive(pff_problem* h, const double* eps3, const double* phi, const double* p3, double* sig3,
                     double* psi, double* tang3) {
    if (!h || !eps3 || !phi) return PFF_ERR_INVALID_ARG;
    const size_t n = h->n();
    int rc;
    for (int j = 0; j < 3; ++j) {
        if ((rc = put_field(h, h->field[5 + j], eps3 + j * n, n, 0))) return rc;
        if (p3) {
            if ((rc = put_field(h, h->field[8 + j], p3 + j * n, n, 0))) return rc;
        } else {
            cudaMemsetAsync(h->field[8 + j], 0, n * (h->prec == PFF_FP64 ? 8 : 4), h->st);
        }
    }
    if ((rc = put_field(h, h->field[18], phi, n, 0))) return rc;
    elem(h, EL_CONSTITUTIVE);
    if ((rc = sync(h, "constitutive"))) return rc;
    for (int j = 0; j < 3; ++j) {
        if (sig3 && (rc = get_field(h, h->field[11 + j], sig3 + j * n, n))) return rc;
        if (tang3 && p3 && (rc = get_field(h, h->field[14 + j], tang3 + j * n, n))) return rc;
    }
    if (psi && (rc = get_field(h, h->field[17], psi, n))) return rc;
    return PFF_OK;
}

int pff_create_batch(int max_slots, size_t hbm_budget, void* cuda_stream, pff_batch** out) {
    if (!out || max_slots < 1) return PFF_ERR_INVALID_ARG;
    pff_batch* b = new pff_batch();
    b->max_slots = max_slots;
    b->budget = hbm_budget;
    b->st = (cudaStream_t)cuda_stream;
    b->slot.assign(max_slots, nullptr);
    *out = b;
    return PFF_OK;
}

int pff_destroy_batch(pff_batch* b) {
    if (!b) return PFF_ERR_INVALID_ARG;
    if (b->st) cudaStreamSynchronize(b->st);
    for (auto& g : b->groups) free_group(g);
    delete b;
    return PFF_OK;
}

int pff_batch_set_group_size(pff_batch* b, int max_problems_per_group) {
    if (!b || max_problems_per_group < 0) return PFF_ERR_INVALID_ARG;
    if (b->st) cudaStreamSynchronize(b->st);
    for (auto& g : b->groups) free_group(g);
    b->groups.clear();
    b->group_cap = max_problems_per_group;
    return PFF_OK;
}

int pff_batch_autotune(pff_batch* b, const int* group_sizes, int n_candidates, int steps_each, int* chosen,
                       pff_step_report* reports, int* steps_done) {
    if (!b || !group_sizes || n_candidates < 1 || steps_each < 1) return PFF_ERR_INVALID_ARG;
    for (int c = 0; c < n_candidates; ++c)
        if (group_sizes[c] < 0) return PFF_ERR_INVALID_ARG;
    const int per = steps_each + 1;              // one untimed step after regrouping (graph capture)
    const int total = n_candidates * per;
    std::vector<int> done(b->max_slots, 0);   // steps run per slot (reports stay contiguous)
    if (steps_done)
        for (int i = 0; i < b->max_slots; ++i) steps_done[i] = 0;
    int status = PFF_OK, best = group_sizes[0];
    double best_score = -1.0;
    for (int c = 0; c < n_candidates; ++c) {
        int rc = pff_batch_set_group_size(b, group_sizes[c]);
        if (rc) return rc;
        double elapsed = 0.0, work = 0.0;
        for (int s = 0; s < per; ++s) {
            std::vector<pff_step_report> one(b->max_slots);
            std::vector<int> d1(b->max_slots, 0);
            const auto t0 = std::chrono::steady_clock::now();
            rc = pff_batch_step(b, 1, one.data(), d1.data());
            const auto t1 = std::chrono::steady_clock::now();
            if (rc && rc != PFF_ERR_NOT_CONVERGED) return rc;
            if (rc) status = rc;
            for (int i = 0; i < b->max_slots; ++i) {
                if (!d1[i]) continue;
                const pff_step_report& r = one[i];
                if (reports) reports[(size_t)i * total + done[i]] = r;
                ++done[i];
                if (s > 0 && b->slot[i])
                    work += (double)(r.mech_cg_iters + r.newton_iters + r.bccg_iters) * b->slot[i]->nx * b->slot[i]->ny;
            }
            if (s > 0) elapsed += std::chrono::duration<double>(t1 - t0).count();
        }
        const double score = elapsed > 0.0 ? work / elapsed : 0.0;
        if (score > best_score) { best_score = score; best = group_sizes[c]; }
    }
    if (steps_done)
        for (int i = 0; i < b->max_slots; ++i) steps_done[i] = done[i];
    int rc = pff_batch_set_group_size(b, best);
    if (rc) return rc;
    if (chosen) *chosen = best;
    return status;
}

int pff_set_kernel_variant(int kind, int grid_n, int ncomp, int variant) {
    if (variant < 0 || variant > 1) return PFF_ERR_INVALID_ARG;
    if (kind == PFF_VARIANT_COLUMN_SHAPE) {
        if (grid_n != 512 || (ncomp != 1 && ncomp != 3)) return PFF_ERR_INVALID_ARG;
        cudaDeviceSynchronize();
        g_col512_cw[ncomp == 3 ? 1 : 0].store(variant == 1 ? 2 : 4);
    } else if (kind == PFF_VARIANT_BCCG_PASSES) {
        cudaDeviceSynchronize();
        g_bccg4.store(variant == 1);
    } else {
        return PFF_ERR_INVALID_ARG;
    }
    g_shape_gen.fetch_add(1);
    return PFF_OK;
}

int pff_get_kernel_variant(int kind, int grid_n, int ncomp, int* variant) {
    if (!variant) return PFF_ERR_INVALID_ARG;
    if (kind == PFF_VARIANT_COLUMN_SHAPE) {
        if (grid_n != 512 || (ncomp != 1 && ncomp != 3)) return PFF_ERR_INVALID_ARG;
        *variant = g_col512_cw[ncomp == 3 ? 1 : 0].load() == 2 ? 1 : 0;
        return PFF_OK;
    }
    if (kind == PFF_VARIANT_BCCG_PASSES) {
        *variant = g_bccg4.load() ? 1 : 0;
        return PFF_OK;
    }
    return PFF_ERR_INVALID_ARG;
}

int pff_batch_autotune_kernels(pff_batch* b, int steps_each, int* chosen, double* scores, pff_step_report* reports,
                               int* steps_done) {
    if (!b || steps_each < 1) return PFF_ERR_INVALID_ARG;
    // candidates: (one-component column shape, three-component column shape, BCCG structure)
    constexpr int NCAND = 8;
    int cand[NCAND][3];
    for (int c = 0; c < NCAND; ++c) { cand[c][0] = c & 1; cand[c][1] = (c >> 1) & 1; cand[c][2] = (c >> 2) & 1; }
    auto apply = [&](int c) {
        int rc = pff_set_kernel_variant(PFF_VARIANT_COLUMN_SHAPE, 512, 1, cand[c][0]);
        if (!rc) rc = pff_set_kernel_variant(PFF_VARIANT_COLUMN_SHAPE, 512, 3, cand[c][1]);
        if (!rc) rc = pff_set_kernel_variant(PFF_VARIANT_BCCG_PASSES, 0, 1, cand[c][2]);
        return rc;
    };
    // steps_each rounds; in each round every candidate runs one untimed load step after its
    // change (graph re-capture) and one timed step, so that all candidates see load steps from
    // the same stretch of the simulations
    const int total = NCAND * 2 * steps_each;
    std::vector<int> done(b->max_slots, 0);
    std::vector<double> elapsed(NCAND, 0.0), work(NCAND, 0.0);
    int status = PFF_OK;
    for (int round = 0; round < steps_each; ++round) {
        for (int cc = 0; cc < NCAND; ++cc) {
            // odd rounds visit the candidates in reverse order, so that a steady drift of the
            // per-iteration cost along the load steps does not favour the early candidates
            const int c = (round & 1) ? NCAND - 1 - cc : cc;
            int rc = apply(c);
            if (rc) return rc;
            for (int s = 0; s < 2; ++s) {
                std::vector<pff_step_report> one(b->max_slots);
                std::vector<int> d1(b->max_slots, 0);
                const auto t0 = std::chrono::steady_clock::now();
                rc = pff_batch_step(b, 1, one.data(), d1.data());
                const auto t1 = std::chrono::steady_clock::now();
                if (rc && rc != PFF_ERR_NOT_CONVERGED) return rc;
                if (rc) status = rc;
                for (int i = 0; i < b->max_slots; ++i) {
                    if (!d1[i]) continue;
                    const pff_step_report& r = one[i];
                    if (reports) reports[(size_t)i * total + done[i]] = r;
                    ++done[i];
                    if (s == 1 && b->slot[i])
                        work[c] += (double)(r.mech_cg_iters + r.newton_iters + r.bccg_iters) * b->slot[i]->nx * b->slot[i]->ny;
                }
                if (s == 1) elapsed[c] += std::chrono::duration<double>(t1 - t0).count();
            }
        }
    }
    int best = 0;
    for (int c = 0; c < NCAND; ++c) {
        const double score = elapsed[c] > 0.0 ? work[c] / elapsed[c] : 0.0;
        if (scores) scores[c] = score;
        if (score > (elapsed[best] > 0.0 ? work[best] / elapsed[best] : 0.0)) best = c;
    }
    if (steps_done)
        for (int i = 0; i < b->max_slots; ++i) steps_done[i] = done[i];
    int rc = apply(best);
    if (rc) return rc;
    if (chosen)
        for (int k = 0; k < 3; ++k) chosen[k] = cand[best][k];
    return status;
}

int pff_batch_admit(pff_batch* b, pff_problem* h, int* slot) {
    if (!b || !h || h->prm.evolution != PFF_NEAR_EQUILIBRIUM) return PFF_ERR_INVALID_ARG;
    for (int i = 0; i < b->max_slots; ++i)
        if (b->slot[i] == h) return PFF_ERR_INVALID_ARG;
    if (b->used + h->bytes > b->budget) return PFF_ERR_OOM;
    for (int i = 0; i < b->max_slots; ++i) {
        if (!b->slot[i]) {
            b->slot[i] = h;
            b->used += h->bytes;
            if (slot) *slot = i;
            return PFF_OK;
        }
    }
    return PFF_ERR_STATE;
}

int pff_batch_release(pff_batch* b, int slot) {
    if (!b || slot < 0 || slot >= b->max_slots || !b->slot[slot]) return PFF_ERR_INVALID_ARG;
    if (b->st) cudaStreamSynchronize(b->st);
    b->used -= b->slot[slot]->bytes;
    b->slot[slot] = nullptr;
    return PFF_OK;
}

int pff_batch_step(pff_batch* b, int n_steps, pff_step_report* reports, int* steps_done) {
    if (!b || n_steps < 0) return PFF_ERR_INVALID_ARG;
    if (steps_done)
        for (int i = 0; i < b->max_slots; ++i) steps_done[i] = 0;
    int status = PFF_OK;
    for (int s = 0; s < n_steps; ++s) {
        int rc = build_groups(b);
        if (rc) return rc;
        if (b->groups.empty()) break;
        const int ng = (int)b->groups.size();
        std::vector<int> rcs(ng, 0);
        // one load step of one group (its own stream when the batch holds several groups)
        auto run_one = [&](int gi) {
            BatchGroup& bg = b->groups[gi];
            pff_problem* h0 = b->slot[bg.slots[0]];
            pff_params p = h0->prm;
            bool energies = false;
            for (int i : bg.slots) {
                const pff_params& q = b->slot[i]->prm;
                p.mech_max_cg = std::max(p.mech_max_cg, q.mech_max_cg);
                p.pf_max_iter = std::max(p.pf_max_iter, q.pf_max_iter);
                p.mech_max_newton = std::max(p.mech_max_newton, q.mech_max_newton);
                energies = energies || q.compute_energies;
            }
            Group g;
            g.nx = bg.nx; g.ny = bg.ny; g.wp = wp_of(bg.nx); g.prec = bg.prec; g.np = (int)bg.slots.size();
            g.st = bg.stream ? bg.stream : b->st;
            g.d_desc = bg.d_desc; g.d_flags = bg.d_flags; g.d_ctrl = bg.d_ctrl;
            g.h_flags = bg.h_flags; g.h_ctrl = bg.h_ctrl; g.graphs = bg.graphs; g.precond = bg.precond;
            rcs[gi] = run_group_step(g, p, energies, h0);
        };
        if (ng == 1) {
            run_one(0);
        } else {
            // the groups' streams start after the caller's stream (copies queued there)
            cudaEvent_t ev = nullptr;
            if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess) {
                cudaEventRecord(ev, b->st);
                for (auto& bg : b->groups)
                    if (bg.stream) cudaStreamWaitEvent(bg.stream, ev, 0);
                cudaEventDestroy(ev);
            }
            std::vector<std::thread> th;
            for (int gi = 0; gi < ng; ++gi) th.emplace_back(run_one, gi);
            for (auto& t : th) t.join();
        }
        for (int gi = 0; gi < ng; ++gi) {
            BatchGroup& bg = b->groups[gi];
            if (rcs[gi]) { b->err = b->slot[bg.slots[0]]->err; return rcs[gi]; }
            for (size_t j = 0; j < bg.slots.size(); ++j) {
                int i = bg.slots[j];
                const Ctrl& c = bg.h_ctrl[j];
                if (reports) fill_report(c, b->slot[i]->split, &reports[(size_t)i * n_steps + s]);
                if (steps_done) steps_done[i] = s + 1;
                if (c.status) status = PFF_ERR_NOT_CONVERGED;
                if (c.broken) b->slot[i]->broken = true;
            }
        }
    }
    return status;
}

unsigned long long pff_kernel_launches(void) { return g_launches.load(); }

int pff_set_graphs(int on) {
    cudaDeviceSynchronize();
    g_graphs_enabled = on != 0;
    g_cond_nodes = on == 2;
    return PFF_OK;
}

int pff_set_persistent(int on) {
    cudaDeviceSynchronize();
    g_persist = on != 0;
    return PFF_OK;
}

int pff_set_cluster_mechanics(int on) {
    cudaDeviceSynchronize();
    g_cluster.store(on != 0);
    return PFF_OK;
}

int pff_set_barrier_spin_limit(long long cycles) {
    if (cycles < 0) return PFF_ERR_INVALID_ARG;
    cudaDeviceSynchronize();
    persist_set_spin(cycles);
    return PFF_OK;
}

int pff_set_pdl(int on) {
    cudaDeviceSynchronize();
    g_pdl.store(on != 0);
    return PFF_OK;
}

int pff_timing_enable(int on) {
    cudaDeviceSynchronize();
    timing_collect();
    g_tm.on = on != 0;
    return PFF_OK;
}

int pff_timing_reset(void) {
    cudaDeviceSynchronize();
    timing_collect();
    std::lock_guard<std::mutex> g(g_tm.mu);
    g_tm.acc.clear();
    return PFF_OK;
}

int pff_timing_read(int family, int op, double* total_ms, unsigned long long* launches) {
    cudaDeviceSynchronize();
    timing_collect();
    std::lock_guard<std::mutex> g(g_tm.mu);
    auto it = g_tm.acc.find(family * 16 + op);
    if (total_ms) *total_ms = it == g_tm.acc.end() ? 0.0 : it->second.first;
    if (launches) *launches = it == g_tm.acc.end() ? 0ull : it->second.second;
    return PFF_OK;
}

}  // extern "C"
