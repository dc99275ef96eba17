// k_persist.cu -- persistent BCCG solve (Sec. 3.1.2, Algorithm 1) for one FP32
// problem of 512 x 512 pixels per launch.
//
// The iterations of the phase-field sub-problem run inside one cooperative
// launch whose blocks all stay resident.  The phases of an iteration -- the
// direction and row FFT pass, the column Laplacian pass, the row-inverse pass
// with J p and its dot products, the elementwise iterate with the residual
// recurrence, and (when a value was clamped, every 32 iterations and to confirm
// convergence) the explicit J v - b chain -- are the same device functions the
// separate kernels use, separated by grid barriers that also carry the
// reductions: each block reduces its share, the last block to arrive sums the
// partials in a fixed order, runs the phase's finalizer (alpha, beta, the
// stopping test) and releases the others.  No kernel boundary remains inside a
// solve.
//
// Every wait is bounded: a block that has not been released after about two
// seconds of clock cycles sets status bit 8 and the abort flag and returns, and
// every other block returns at its next barrier.  Global loads of this
// translation unit bypass L1 (-Xptxas -dlcm=cg at build), since L1 is not
// coherent between the SMs within one kernel; spectrum rows are staged with
// 16-byte-or-wider copies only where they are coherent (plain loads here).
#include <atomic>

#include "kernels.cuh"
#include "launch.h"

namespace pff {
namespace {

constexpr int PB_NT = 128;                        // threads per block (the FP32 512-row pass geometry)
constexpr int PB_CW = 2;                          // columns per column item (64 threads each)
constexpr long long PB_SPIN_CYCLES = 4000000000LL;   // default wait limit of a barrier (about two seconds)

using RC = RowCfg<float, 512, 1>;
static_assert(RC::NT == PB_NT && RC::ROWS == 2, "row geometry of the persistent kernel");

__device__ __forceinline__ unsigned ld_volatile(const unsigned* p) { return *(const volatile unsigned*)p; }
__device__ __forceinline__ int ld_volatile(const int* p) { return *(const volatile int*)p; }

// Grid barrier with an optional reduction of NR values (double-float within the
// block, FP64 across blocks).  A block waits at most `spin` clock cycles for the
// release.  Returns false in every thread after a timeout or an abort.
template <int NR, class FIN>
__device__ bool grid_sync(Ctrl* c, double* part, DF (&v)[NR > 0 ? NR : 1], FIN fin, long long spin) {
    using O = RedOps<DF>;
    constexpr int NW = PB_NT / 32;
    constexpr int NRA = NR > 0 ? NR : 1;
    __shared__ DF sh[NRA][NW];
    __shared__ int s_last, s_ok;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if constexpr (NR > 0) {
#pragma unroll
        for (int k = 0; k < NR; ++k) {
            DF x = v[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x = O::add(x, O::shfl(x, o));
            if (lane == 0) sh[k][warp] = x;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned gen = ld_volatile(&c->bar_gen);
        if constexpr (NR > 0) {
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                DF x = sh[k][0];
                for (int w = 1; w < NW; ++w) x = O::add(x, sh[k][w]);
                __stcg(part + (size_t)blockIdx.x * NR + k, O::total(x));   // FP64 block total
            }
        }
        __threadfence();
        const unsigned t = atomicAdd(&c->bar_count, 1u);
        s_last = (t == gridDim.x - 1);
        s_ok = 1;
        if (!s_last) {
            const long long t0 = clock64();
            while (ld_volatile(&c->bar_gen) == gen) {
                if (ld_volatile(&c->bar_abort) || clock64() - t0 > spin) { s_ok = 0; break; }
                __nanosleep(32);
            }
            __threadfence();
        }
    }
    __syncthreads();
    if (s_last) {
        double tot[NRA];
        __shared__ double shd[NRA][NW];
        if constexpr (NR > 0) {
            // FP64 cross-block sum in a fixed order
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                double x = 0.0;
                for (int b = threadIdx.x; b < (int)gridDim.x; b += PB_NT) x += __ldcg(part + (size_t)b * NR + k);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
                if (lane == 0) shd[k][warp] = x;
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            if constexpr (NR > 0) {
#pragma unroll
                for (int k = 0; k < NR; ++k) {
                    double x = shd[k][0];
                    for (int w = 1; w < NW; ++w) x += shd[k][w];
                    tot[k] = x;
                }
            }
            fin(tot);
            c->bar_count = 0u;
            __threadfence();
            atomicAdd(&c->bar_gen, 1u);   // release
        }
        __syncthreads();
    }
    if (!s_ok) {
        if (threadIdx.x == 0) {
            atomicOr(&c->status, 8);
            atomicExch(&c->bar_abort, 1);
        }
        return false;
    }
    return true;
}

// F's per-block constants evaluated by thread 0 (after a barrier) and shared
template <class F>
__device__ __forceinline__ typename F::Ctx bcast_prep(const Desc<float>& d) {
    using X = typename F::Ctx;
    __shared__ __align__(16) unsigned char raw[sizeof(X)];
    __syncthreads();
    if (threadIdx.x == 0) {
        const X c = F::prep(d);
        memcpy(raw, &c, sizeof(X));
    }
    __syncthreads();
    X c;
    memcpy(&c, raw, sizeof(X));
    return c;
}

struct NoFin {
    __device__ void operator()(const double*) const {}
};

template <class F>
struct Fin {
    const Desc<float>& d;
    __device__ void operator()(const double* tot) const { F::finalize(d, tot); }
};

// Phases are compiled as separate (not inlined) functions so that the kernel's
// register allocation is that of the largest phase, not of their union.
template <class F>
__device__ __noinline__ bool row_fwd_phase(const Desc<float>& d, float2* work, const float2* rtw, long long spin) {
    const typename F::Ctx ctx = bcast_prep<F>(d);
    Acc<float> acc[1];
    for (int item = blockIdx.x; item < 512 / RC::ROWS; item += gridDim.x) {
        __syncthreads();
        row_fwd_pixels<float, 512, 1, F>(d, ctx, item * RC::ROWS, work, &acc[0]);
        __syncthreads();
        row_fwd_fft_store<float, 512, 1>(d, item * RC::ROWS, work, rtw);
    }
    DF none[1];
    return grid_sync<0>(d.ctrl, d.part, none, NoFin{}, spin);
}

template <class OP>
__device__ __noinline__ bool col_phase(const Desc<float>& d, float2* work, const float2* ctw, long long spin) {
    const ModeK<float> mk(d);
    for (int item = blockIdx.x; item < (d.nx / 2 + PB_CW) / PB_CW; item += gridDim.x) {   // mode columns only
        __syncthreads();
        col512_item<float, 1, OP, PB_CW>(d, mk, item * PB_CW, work, ctw);
    }
    DF none[1];
    return grid_sync<0>(d.ctrl, d.part, none, NoFin{}, spin);
}

template <class F>
__device__ __noinline__ bool row_inv_phase(const Desc<float>& d, float2* work, const float2* rtw, long long spin) {
    const typename F::Ctx ctx = bcast_prep<F>(d);
    Acc<float> acc[F::NR];
    for (int item = blockIdx.x; item < 512 / RC::ROWS; item += gridDim.x) {
        __syncthreads();
        row_inv_item<float, 512, 1, F>(d, ctx, item * RC::ROWS, work, rtw, &acc[0]);
    }
    DF v[F::NR];
#pragma unroll
    for (int k = 0; k < F::NR; ++k) v[k] = acc[k].df();
    return grid_sync<F::NR>(d.ctrl, d.part, v, Fin<F>{d}, spin);
}

template <class F>
__device__ __noinline__ bool elem_phase(const Desc<float>& d, long long spin) {
    const typename F::Ctx ctx = bcast_prep<F>(d);
    Acc<float> acc[F::NR];
    elem_items<float, F>(d, ctx, &acc[0]);
    DF v[F::NR];
#pragma unroll
    for (int k = 0; k < F::NR; ++k) v[k] = acc[k].df();
    return grid_sync<F::NR>(d.ctrl, d.part, v, Fin<F>{d}, spin);
}

constexpr int PB_WORK = RC::NSEQ * RC::SP > PB_CW * COL512_XS ? RC::NSEQ * RC::SP : PB_CW * COL512_XS;
constexpr size_t PB_SMEM = (size_t)(RC::TWS + padded_len(512) + PB_WORK) * sizeof(float2);

__global__ void __launch_bounds__(PB_NT, 4) k_bccg512(const Desc<float>* __restrict__ descs, int max_iters,
                                                        long long spin) {
    const Desc<float>& d = descs[0];
    Ctrl* c = d.ctrl;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* rtw = reinterpret_cast<float2*>(smem_raw);
    float2* ctw = rtw + RC::TWS;
    float2* work = ctw + padded_len(512);
    stage_row_twiddles<float, 512, 1>(d, rtw);
    stage_col512_twiddles<float>(d, ctw);
    cp_async_wait_all();
    __syncthreads();
    for (int it = 0; it <= max_iters; ++it) {
        if (__ldcg(&c->pf_b) || ld_volatile(&c->bar_abort)) break;   // the same decision in every block
        if (!row_fwd_phase<FPfA1<float>>(d, work, rtw, spin)) return;
        if (!col_phase<FColLapPF>(d, work, ctw, spin)) return;
        if (!row_inv_phase<FPfA3<float>>(d, work, rtw, spin)) return;
        if (!elem_phase<FPfB1<float>>(d, spin)) return;
        if (__ldcg(&c->pf_full)) {
            if (!row_fwd_phase<FPfVIn<float>>(d, work, rtw, spin)) return;
            if (!col_phase<FColLapPFFull>(d, work, ctw, spin)) return;
            if (!row_inv_phase<FPfB3<float>>(d, work, rtw, spin)) return;
        }
    }
}

}  // namespace

// Blocks of the persistent launch: all resident at once (cooperative launch),
// at most `share` of the device's resident capacity, at most one per row item.
int persist_bccg_blocks(int share_den) {
    static int cap = -1;
    if (cap < 0) {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncSetAttribute(k_bccg512, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PB_SMEM);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_bccg512, PB_NT, PB_SMEM);
        cap = per * sms;
        cudaGetLastError();
    }
    int b = cap / (share_den > 0 ? share_den : 1);
    if (b > 512 / RC::ROWS) b = 512 / RC::ROWS;
    return b;
}

// Wait limit of the grid barriers in clock cycles (0: the default of about two seconds).
static std::atomic<long long> g_spin{0};
void persist_set_spin(long long cycles) { g_spin.store(cycles > 0 ? cycles : 0); }

// Launches the persistent solve of one FP32 512 x 512 problem (after its BCCG start).
cudaError_t launch_persist_bccg(const Desc<float>* d, int max_iters, int blocks, cudaStream_t st) {
    if (blocks < 1) return cudaErrorInvalidConfiguration;
    long long spin = g_spin.load();
    if (spin <= 0) spin = PB_SPIN_CYCLES;
    void* args[] = {(void*)&d, (void*)&max_iters, (void*)&spin};
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_bccg512, dim3(blocks), dim3(PB_NT), args, PB_SMEM, st);
    count_launch();
    return e;
}

}  // namespace pff
