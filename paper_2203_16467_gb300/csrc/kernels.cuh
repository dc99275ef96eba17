// kernels.cuh -- elementwise kernels, the driving-force maximum (Algorithm 4
// lines 4-10) and the launch dispatch by grid size.
#pragma once
#include "ops.cuh"
#include "launch.h"

namespace pff {

constexpr int EL_NT = 256;

// Elementwise work of functor F over the problem's pixels, grid-stride over the
// launch's blocks (accumulating F's reductions in acc).
template <typename T, class F>
__device__ __forceinline__ void elem_items(const Desc<T>& d, const typename F::Ctx& ctx, Acc<T>* acc) {
    // 32-bit pixel indices (grids have fewer than 2^32 pixels), widened at the access
    const unsigned n = (unsigned)d.nx * d.ny;
    const unsigned stride = gridDim.x * blockDim.x;
    if constexpr (HasIn<F>::value) {
        constexpr int U = 4;   // pixels whose loads are in flight together
        for (unsigned base = blockIdx.x * blockDim.x + threadIdx.x; base < n; base += U * stride) {
            typename F::In in[U];
#pragma unroll
            for (int j = 0; j < U; ++j)
                if (base + j * stride < n) in[j] = F::load(d, ctx, (size_t)(base + j * stride));
#pragma unroll
            for (int j = 0; j < U; ++j)
                if (base + j * stride < n) F::pixel(d, ctx, (size_t)(base + j * stride), in[j], acc);
        }
    } else {
        for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) F::pixel(d, ctx, (size_t)i, acc);
    }
}

template <typename T, class F>
__global__ void __launch_bounds__(EL_NT) k_elem(const Desc<T>* __restrict__ descs) {
    const Desc<T>& d = descs[blockIdx.y];
    pdl_enter();
    typename F::Ctx ctx;
    if (block_prep<F>(d, ctx)) return;
    constexpr int NRA = F::NR > 0 ? F::NR : 1;
    Acc<T> acc[NRA];
    elem_items<T, F>(d, ctx, &acc[0]);
    if constexpr (F::NR > 0) {
        double tot[F::NR];
        if (reduce_acc<F::NR, EL_NT>(acc, d.part, &d.ctrl->counter, gridDim.x, tot) && threadIdx.x == 0)
            F::finalize(d, tot);
    }
}

// Reset of the per-step solver state (one thread per problem).
template <typename T>
__global__ void k_step_begin(const Desc<T>* __restrict__ descs, int np) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= np) return;
    Ctrl* c = descs[j].ctrl;
    c->nd_a = 0; c->nd_b = 0; c->newton_it = 0; c->needs_fold = 0;
    c->cg_a = 1; c->cg_b = 1; c->cg_it = 0; c->cg_total = 0; c->cg_break = 0;
    c->pf_a = 1; c->pf_b = 1; c->pf_it = 0; c->pf_break = 0; c->n_active = 0; c->pf_clamp_iters = 0;
    c->gamma = 1.0; c->rescaled = 0; c->status = 0; c->counter = 0u;
    c->Ff = 0.0;
}

// Solver flags of every problem of a group: bit0 CG done, bit1 Newton done, bit2 BCCG done.
template <typename T>
__global__ void k_gather(const Desc<T>* __restrict__ descs, int np, int* out) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= np) return;
    const Ctrl* c = descs[j].ctrl;
    out[j] = (__ldcg(&c->cg_b) ? 1 : 0) | (__ldcg(&c->nd_a) ? 2 : 0) | (__ldcg(&c->pf_b) ? 4 : 0);
}

// -F_phi = D + R_f with D = 2(1-phi) psi_0^+ and R_f = -c (f'(phi) - 2 ell^2 lap phi),
// evaluated in FP64; first maximiser in row-major order; max D; then the
// rescale decision of Algorithm 4 lines 4-10 (readings in the oracle docs).
struct ArgMax {
    double v, D, R, Dmax;
    long long i;
};
__device__ __forceinline__ void am_merge(ArgMax& a, const ArgMax& b) {
    if (b.v > a.v || (b.v == a.v && b.i < a.i)) { a.v = b.v; a.i = b.i; a.D = b.D; a.R = b.R; }
    a.Dmax = fmax(a.Dmax, b.Dmax);
}
__device__ __forceinline__ ArgMax am_shfl(const ArgMax& a, int o) {
    ArgMax b;
    b.v = __shfl_down_sync(0xffffffffu, a.v, o);
    b.D = __shfl_down_sync(0xffffffffu, a.D, o);
    b.R = __shfl_down_sync(0xffffffffu, a.R, o);
    b.Dmax = __shfl_down_sync(0xffffffffu, a.Dmax, o);
    b.i = __shfl_down_sync(0xffffffffu, a.i, o);
    return b;
}

template <typename T>
__global__ void __launch_bounds__(EL_NT) k_df(const Desc<T>* __restrict__ descs) {
    const Desc<T>& d = descs[blockIdx.y];
    const Consts& k = d.k;
    Ctrl* ctrl = d.ctrl;
    double eb[3];
    for (int j = 0; j < 3; ++j) eb[j] = ldd(&ctrl->eps_bar[j]);
    ArgMax best{-INFINITY, 0.0, 0.0, -INFINITY, 0x7fffffffffffffffLL};
    const size_t n = (size_t)d.nx * d.ny;
    for (size_t i = (size_t)blockIdx.x * EL_NT + threadIdx.x; i < n; i += (size_t)gridDim.x * EL_NT) {
        double E = (double)d.E[i];
        double psi = psi_plus<double>(k.split, eb[0] + (double)d.eps[0][i], eb[1] + (double)d.eps[1][i],
                                      eb[2] + (double)d.eps[2][i], k.lam_c * E, k.mu_c * E);
        double ph = (double)d.phi[i];
        double D = 2.0 * (1.0 - ph) * psi;
        double fp = k.fracture == AT1 ? 1.0 : 2.0 * ph;
        double R = -k.c * fp + k.kappa * (double)d.lap[i];
        double v = D + R;
        if (v > best.v) { best.v = v; best.i = (long long)i; best.D = D; best.R = R; }
        best.Dmax = fmax(best.Dmax, D);
    }
    __shared__ ArgMax sh[EL_NT / 32];
    __shared__ int s_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) { ArgMax b = am_shfl(best, o); am_merge(best, b); }
    if (lane == 0) sh[warp] = best;
    __syncthreads();
    double* part = d.part;
    if (threadIdx.x == 0) {
        ArgMax a = sh[0];
        for (int w = 1; w < EL_NT / 32; ++w) am_merge(a, sh[w]);
        size_t o = (size_t)blockIdx.x * 5;
        __stcg(&part[o + 0], a.v); __stcg(&part[o + 1], a.D); __stcg(&part[o + 2], a.R);
        __stcg(&part[o + 3], a.Dmax); __stcg(&part[o + 4], (double)a.i);
        __threadfence();
        unsigned t = atomicAdd(&ctrl->counter, 1u);
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last || threadIdx.x != 0) return;
    __threadfence();
    ArgMax a{-INFINITY, 0.0, 0.0, -INFINITY, 0x7fffffffffffffffLL};
    for (unsigned b = 0; b < gridDim.x; ++b) {
        ArgMax c{__ldcg(&part[b * 5 + 0]), __ldcg(&part[b * 5 + 1]), __ldcg(&part[b * 5 + 2]),
                 __ldcg(&part[b * 5 + 3]), (long long)__ldcg(&part[b * 5 + 4])};
        am_merge(a, c);
    }
    ctrl->counter = 0u;
    ctrl->mF_max = a.v;
    ctrl->D_max = a.Dmax;
    ctrl->istar = (int)a.i;
    ctrl->Rf_star = a.R;
    ctrl->D_star = a.D;
    if (a.v > k.Fmax && a.Dmax > k.thresh) ctrl->flag = 1;
    double g = 1.0;
    if (a.v > k.Fmax && ctrl->flag) {
        double num = k.Fmax - a.R, den = a.D;
        if (num > 0.0 && den > 0.0) {
            g = sqrt(num / den);
            double em = fmax(fmax(fabs(eb[0]), fabs(eb[1])), fabs(eb[2]));
            double dm = fmax(fmax(fabs(k.d_eps_bar[0]), fabs(k.d_eps_bar[1])), fabs(k.d_eps_bar[2]));
            if (em > 0.0) g = fmin(g, 1.0 + dm / em);
        }
    }
    ctrl->gamma = g;
    ctrl->rescaled = g != 1.0;
}

// ---- field evaluation for the operator entry points and pff_get_fields
// constitutive entry: eps in th[], phi in aux, p in r[] -> sigma in p[], psi_0^+ in lap, C:p in q[]
template <typename T>
struct FConstitutive {
    static constexpr int NR = 0;
    using Ctx = NoCtx;
    __device__ static bool skip(const Desc<T>&) { return false; }
    __device__ static Ctx prep(const Desc<T>&) { return Ctx{}; }
    __device__ static void pixel(const Desc<T>& d, const Ctx&, size_t i, Acc<T>*) {
        T lam, mu;
        lame_at(d, i, lam, mu);
        T xx = d.th[0][i], yy = d.th[1][i], xy = d.th[2][i];
        T h = hdeg(d.aux[i]);
        T s[3], t[3];
        stress(d.k.split, xx, yy, xy, h, lam, mu, s);
        tangent(d.k.split, xx, yy, xy, h, lam, mu, d.r[0][i], d.r[1][i], d.r[2][i], t);
        for (int k = 0; k < 3; ++k) { d.p[k][i] = s[k]; d.q[k][i] = t[k]; }
        d.lap[i] = psi_plus(d.k.split, xx, yy, xy, lam, mu);
    }
    __device__ static void finalize(const Desc<T>&, const double*) {}
};

// state fields: sigma(eps_bar + eps*, phi) -> q[], psi_0^+ -> aux
template <typename T>
struct FStateFields {
    static constexpr int NR = 0;
    struct Ctx { T eb[3]; };
    __device__ static bool skip(const Desc<T>&) { return false; }
    __device__ static Ctx prep(const Desc<T>& d) {
        Ctx c;
        for (int k = 0; k < 3; ++k) c.eb[k] = T(ldd(&d.ctrl->eps_bar[k]));
        return c;
    }
    __device__ static void pixel(const Desc<T>& d, const Ctx& c, size_t i, Acc<T>*) {
        T lam, mu;
        lame_at(d, i, lam, mu);
        T xx = c.eb[0] + d.eps[0][i], yy = c.eb[1] + d.eps[1][i], xy = c.eb[2] + d.eps[2][i];
        T s[3];
        stress(d.k.split, xx, yy, xy, hdeg(d.phi[i]), lam, mu, s);
        for (int k = 0; k < 3; ++k) d.q[k][i] = s[k];
        d.aux[i] = psi_plus(d.k.split, xx, yy, xy, lam, mu);
    }
    __device__ static void finalize(const Desc<T>&, const double*) {}
};

// -F_phi field (needs lap = nabla^2 phi): into p[0]
template <typename T>
struct FDrivingField {
    static constexpr int NR = 0;
    struct Ctx { double eb[3]; };
    __device__ static bool skip(const Desc<T>&) { return false; }
    __device__ static Ctx prep(const Desc<T>& d) {
        Ctx c;
        for (int k = 0; k < 3; ++k) c.eb[k] = ldd(&d.ctrl->eps_bar[k]);
        return c;
    }
    __device__ static void pixel(const Desc<T>& d, const Ctx& c, size_t i, Acc<T>*) {
        const Consts& k = d.k;
        double E = (double)d.E[i];
        double psi = psi_plus<double>(k.split, c.eb[0] + (double)d.eps[0][i], c.eb[1] + (double)d.eps[1][i],
                                      c.eb[2] + (double)d.eps[2][i], k.lam_c * E, k.mu_c * E);
        double ph = (double)d.phi[i];
        double fp = k.fracture == AT1 ? 1.0 : 2.0 * ph;
        d.p[0][i] = T(2.0 * (1.0 - ph) * psi - k.c * fp + k.kappa * (double)d.lap[i]);
    }
    __device__ static void finalize(const Desc<T>&, const double*) {}
};

template <typename T>
struct FFlagsField {   // active flag -> p[1]
    static constexpr int NR = 0;
    using Ctx = NoCtx;
    __device__ static bool skip(const Desc<T>&) { return false; }
    __device__ static Ctx prep(const Desc<T>&) { return Ctx{}; }
    __device__ static void pixel(const Desc<T>& d, const Ctx&, size_t i, Acc<T>*) {
        d.p[1][i] = (d.flags[i] & 2) ? T(1) : T(0);
    }
    __device__ static void finalize(const Desc<T>&, const double*) {}
};

// ---------------------------------------------------------------------------
// launch helpers
void count_launch();
void note_launch_error(cudaError_t e);   // reported by the next poll of this host thread
bool pdl_on();   // launch the operator kernels with programmatic stream serialization

// Launch of a kernel that begins with pdl_enter() (row, column and elementwise
// kernels): with the attribute it may be scheduled while its predecessor runs.
// Only FP32 kernels use it: FP64 kernels measured slower with it.
template <typename T, typename... P, typename... A>
inline void launch_pdl(void (*fn)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, A... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = (sizeof(T) == 4 && pdl_on()) ? 1 : 0;
    cudaError_t e = cudaLaunchKernelEx(&cfg, fn, args...);
    if (e != cudaSuccess) note_launch_error(e);
}
bool smem_optin(const void* fn, size_t smem);
// columns per block of the 512-point FP32 column pass with nc components (4 or 2; see pff_set_fft_variant)
int col512_cw(int nc);
// optional per-kernel-class event timing (see pff_timing_enable); key = family * 16 + op
bool timing_on();
void timing_begin(int key, cudaStream_t st);
void timing_end(int key, cudaStream_t st);
enum { FAM_ROW_FWD = 0, FAM_ROW_INV = 1, FAM_COL = 2, FAM_ELEM = 3, FAM_CLUSTER = 4 };

template <typename T, int NX, int NC, class F>
void go_row_fwd(const Desc<T>* d, int np, int ny, cudaStream_t st, int key) {
    using Cfg = RowCfg<T, NX, NC>;
    void (*fn)(const Desc<T>*);
    if constexpr (Cfg::MINB > 1) fn = k_row_fwd<T, NX, NC, F>;
    else fn = k_row_fwd_u<T, NX, NC, F>;
    smem_optin((const void*)fn, Cfg::SMEM);
    const bool tm = timing_on();
    if (tm) timing_begin(key, st);
    launch_pdl<T>(fn, dim3(ny / Cfg::ROWS, np), dim3(Cfg::NT), Cfg::SMEM, st, d);
    if (tm) timing_end(key, st);
    count_launch();
}
template <typename T, int NX, int NC, class F>
void go_row_inv(const Desc<T>* d, int np, int ny, cudaStream_t st, int key) {
    using Cfg = RowCfg<T, NX, NC>;
    void (*fn)(const Desc<T>*);
    if constexpr (Cfg::MINB_INV > 1) fn = k_row_inv<T, NX, NC, F>;
    else fn = k_row_inv_u<T, NX, NC, F>;
    smem_optin((const void*)fn, Cfg::SMEM);
    const bool tm = timing_on();
    if (tm) timing_begin(key, st);
    launch_pdl<T>(fn, dim3(ny / Cfg::ROWS, np), dim3(Cfg::NT), Cfg::SMEM, st, d);
    if (tm) timing_end(key, st);
    count_launch();
}
// nm = nx/2 + 1 mode columns: ceil(nm / columns per block) blocks per problem
template <typename T, int NY, int NC, class OP>
void go_col(const Desc<T>* d, int np, int nm, cudaStream_t st, int key) {
    const bool tm = timing_on();
    if (tm) timing_begin(key, st);
    if constexpr (NY == 512 && sizeof(T) == 4) {   // register-resident radix-8 stages (FP64: too many registers)
        if (col512_cw(NC) == 2) {   // shape variant: 2 columns (128 threads) per block
            using Cfg = Col512Cfg<T, NC, 2>;
            auto fn = k_col512<T, NC, OP, 2>;
            smem_optin((const void*)fn, Cfg::SMEM);
            launch_pdl<T>(fn, dim3((nm + 1) / 2, np), dim3(Cfg::NT), Cfg::SMEM, st, d);
        } else {
            using Cfg = Col512Cfg<T, NC, COL512_CW>;
            auto fn = k_col512<T, NC, OP, COL512_CW>;
            smem_optin((const void*)fn, Cfg::SMEM);
            launch_pdl<T>(fn, dim3((nm + COL512_CW - 1) / COL512_CW, np), dim3(Cfg::NT), Cfg::SMEM, st, d);
        }
    } else {
        using Cfg = ColCfg<T, NY, NC>;
        auto fn = k_col<T, NY, NC, OP>;
        smem_optin((const void*)fn, Cfg::SMEM);
        launch_pdl<T>(fn, dim3((nm + Cfg::CWE - 1) / Cfg::CWE, np), dim3(Cfg::NT), Cfg::SMEM, st, d);
    }
    if (tm) timing_end(key, st);
    count_launch();
}

#define PFF_SIZE_SWITCH(n, CALL)                    \
    switch (n) {                                    \
        case 16: { constexpr int N_ = 16; CALL; } break;     \
        case 32: { constexpr int N_ = 32; CALL; } break;     \
        case 64: { constexpr int N_ = 64; CALL; } break;     \
        case 128: { constexpr int N_ = 128; CALL; } break;   \
        case 256: { constexpr int N_ = 256; CALL; } break;   \
        case 512: { constexpr int N_ = 512; CALL; } break;   \
        case 1024: { constexpr int N_ = 1024; CALL; } break; \
        case 2048: { constexpr int N_ = 2048; CALL; } break; \
        default: break;                             \
    }

inline int elem_blocks(int nx, int ny, int np) {
    long long n = (long long)nx * ny;
    long long b = (n + EL_NT * 4 - 1) / (EL_NT * 4);
    long long cap = 2048;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    (void)np;
    return (int)b;
}

}  // namespace pff
