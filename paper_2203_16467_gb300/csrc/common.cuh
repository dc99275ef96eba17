// common.cuh -- device data layout, per-problem control block, pointwise
// constitutive model (Sec. 2.1) and deterministic reductions shared by every
// kernel of libpff.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pff {

// ---------------------------------------------------------------------------
// complex helpers
template <typename T> struct CT;
template <> struct CT<float> { using t = float2; };
template <> struct CT<double> { using t = double2; };

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) { return C{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
// a * conj(b)
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) { return C{a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y}; }

// model enums (mirror include/pff.h)
enum { AT1 = 1, AT2 = 2 };
enum { ISOTROPIC = 0, SPECTRAL = 1, SPECTRAL_STRESSFREE = 2, VOLDEV = 3, SPECTRAL_VOLDEV = 4 };
// split that supplies the stress (contact model) / the crack driving force (Sec. 2.1, Sec. 4.2)
__host__ __device__ __forceinline__ int contact_of(int split) {
    return split == SPECTRAL_STRESSFREE ? ISOTROPIC : (split == SPECTRAL_VOLDEV ? VOLDEV : split);
}
__host__ __device__ __forceinline__ int driving_of(int split) {
    return (split == SPECTRAL_STRESSFREE || split == SPECTRAL_VOLDEV) ? SPECTRAL : split;
}
enum { CRACK_SET = 0, DAMAGE = 1 };

// ---------------------------------------------------------------------------
// Control block of one problem (device memory).  Scalars of the iterative
// solvers live here so that kernels chain without host round trips.  Flags
// come in pairs (x_a, x_b): a kernel never writes a flag that kernels of the
// same launch read, so early-exit decisions are consistent across its blocks.
struct Ctrl {
    // macroscopic strain and loading
    double eps_bar[3];
    double sumE2;           // sum of E^2 over pixels (scale of the mechanics tolerance)
    double sumE;            // sum of E
    // mechanics
    double mech_target, R2, rr, pAp, rAp, qq, alpha, beta, cg_target;
    int nd_a, nd_b, newton_it, needs_fold;
    int cg_a, cg_b, cg_it, cg_total, cg_break;
    // near-equilibrium rescale (Algorithm 4 lines 4-10)
    double mF_max, D_max, Rf_star, D_star, gamma;
    int istar, flag, rescaled;
    // phase field (Algorithm 1)
    double pf_rr, pf_rp, pJp, pf_alpha, pf_beta, pf_target, pf_best;
    double pf_pap;          // sum a p^2 of the direction (the diagonal part of p.Jp)
    int pf_a, pf_b, pf_it, pf_break, n_active, pf_best_it, pf_clamp_iters;
    // residual recurrence: pf_full = this iteration evaluates Jv explicitly
    int pf_full, pf_force, pf_confirm, pf_since_full, pf_full_iters;
    int pf_rsel;            // the BCCG residual r lives in th[1] (0) or q[1] (1)
    double pf_abar;         // mean of the BCCG diagonal a (preconditioner)
    double pf_rz;           // r.z of the previous preconditioned iteration
    // grid barrier of the persistent BCCG kernel (arrivals, release generation, abort)
    unsigned bar_count, bar_gen;
    int bar_abort;
    double pf_last_full;
    // post-step (Algorithm 4 lines 12-14)
    double rep_eps_bar[3], sig_bar[3], C_bar, dphi, Fe, Ff;
    int incremented, broken;
    int status;             // bit0: mechanics cap hit, bit1: BCCG cap hit
    unsigned counter;       // last-block reduction counter (reset by the last block)
    // set by the host for the alternating-minimisation / time-dependent methods
    double eta_dt_override; // eta/dt of the phase-field step when use_override
    int use_override;
    int con_frozen;         // constraint field phi_con taken from aux (fixed over an increment)
    int post_mode;          // 0: post-step applies Algorithm 4's strain increment; 1: host decides
    int pad;
};

// Model constants of a problem, resolved on the host.
struct Consts {
    double lam_c, mu_c;     // lambda = lam_c * E, mu = mu_c * E (plane strain)
    double c;               // G_c / (c_w ell)
    double kappa;           // 2 c ell^2 (coefficient of -nabla^2 in J)
    double ell2;            // ell^2
    double eta_dt;          // eta / dt
    double cf2;             // c * f''
    double Fmax, thresh, dphi_min, C_broken, crack_thr;
    double mech_tol, mech_cg_rtol, pf_tol, pf_atol, pf_floor;
    double d_eps_bar[3];
    double dA;              // pixel area
    double inv_n;           // 1 / (nx ny)
    double L1_scale;        // (dx/ell)^2
    double two_pi_over_Lx, two_pi_over_Ly;
    double lp_a, lp_b, lp_c;  // low-pass band kx^2 lp_a + ky^2 lp_b <= lp_c (microstructure generator only)
    int max_newton, max_cg, max_pf;
    int pf_precond;         // BCCG with the Fourier Helmholtz preconditioner
    int fracture, split, irrev;
};

// Device descriptor of one problem's fields (all arrays nx*ny, row-major).
// Phase-field work vectors alias the mechanics CG vectors:
//   v = th[0], rb = th[1], pb = th[2], a = r[0], b = r[1], vcon = r[2].
template <typename T>
struct Desc {
    using C = typename CT<T>::t;
    T* E;
    T* phi;
    T* eps[3];
    T* th[3];
    T* r[3];
    T* p[3];
    T* q[3];
    T* lap;
    T* aux;
    uint8_t* flags;
    C* S;                   // spectral buffer [3][ny][wp]
    const C* tw;            // twiddle tables of this device
    double* part;           // reduction partials [blocks * 8]
    Ctrl* ctrl;
    int nx, ny, wp, pad;
    Consts k;
};

// ---------------------------------------------------------------------------
// Programmatic dependent launch: a kernel's blocks may be scheduled while the
// previous kernel of the stream is still running; they do only work on
// immutable data (descriptor, twiddle tables) before pdl_wait(), which returns
// once the previous kernel has completed and its writes are visible.  Each
// kernel then lets the next one be scheduled.  Both are no-ops for launches
// without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_enter() { pdl_wait(); pdl_release(); }

// ---------------------------------------------------------------------------
// Per-block constants: thread 0 evaluates F::skip and F::prep once (control
// block loads and FP64-to-FP32 conversions, which run on GB300's narrow FP64
// pipe) and shares the result through shared memory.  Returns true when the
// whole problem is skipped.  Ctx must be trivially copyable.
template <class F, class D, class X>
__device__ __forceinline__ bool block_prep(const D& d, X& ctx) {
    __shared__ __align__(16) unsigned char s_raw[sizeof(X)];
    __shared__ int s_skip;
    if (threadIdx.x == 0) {
        s_skip = F::skip(d) ? 1 : 0;
        if (!s_skip) {
            const X c = F::prep(d);
            memcpy(s_raw, &c, sizeof(X));
        }
    }
    __syncthreads();
    if (s_skip) return true;
    memcpy(&ctx, s_raw, sizeof(X));
    return false;
}

// ---------------------------------------------------------------------------
// flag access (bypass L1: flags are written by other kernels / blocks)
__device__ __forceinline__ int ldflag(const int* p) { return __ldcg(p); }
__device__ __forceinline__ double ldd(const double* p) { return __ldcg(p); }

// ---------------------------------------------------------------------------
// Per-thread accumulation.  FP64 problems accumulate in double.  FP32 problems
// accumulate products exactly split (fmaf) and summed with Knuth's two-sum in
// a float pair, and reduce across the grid in double-float arithmetic
// (reduce_grid): the work stays on the FP32 pipe while the sums keep close to
// FP64 accuracy.
// Functors whose per-pixel work splits into load() (returning an In record) and
// pixel(..., const In&, ...) let a kernel issue the loads of all of a thread's
// pixels before the first store, so that they are in flight together.
template <class F, class = void> struct HasIn { static constexpr bool value = false; };
template <class F> struct HasIn<F, decltype((void)sizeof(typename F::In), void())> { static constexpr bool value = true; };

template <class F, class D, class X, class... A>
__device__ __forceinline__ void pixel_one(const D& d, const X& c, size_t i, A&&... a) {
    if constexpr (HasIn<F>::value) F::pixel(d, c, i, F::load(d, c, i), a...);
    else F::pixel(d, c, i, a...);
}

struct DF { float hi, lo; };   // double-float value hi + lo (see reduce_grid)
template <typename T> struct Acc;
// count(x): a small integer (a pixel count); a thread's sum of counts is exact in
// either precision (below 2^24), so it needs no compensation.
template <> struct Acc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ void count(double x) { s += x; }
    __device__ __forceinline__ void addp(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ double get() const { return s; }
};
template <> struct Acc<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void count(float x) { s += x; }
    __device__ __forceinline__ void add(float x) {
        float t = s + x;
        float z = t - s;
        c += (s - (t - z)) + (x - z);
        s = t;
    }
    __device__ __forceinline__ void addp(float a, float b) {
        float pr = __fmul_rn(a, b);   // not contracted into the two-sum below
        float e = fmaf(a, b, -pr);
        add(pr);
        c += e;
    }
    __device__ __forceinline__ double get() const { return (double)s + (double)c; }
    __device__ __forceinline__ DF df() const {   // normalised double-float pair
        float h = s + c;
        float z = h - s;
        return DF{h, (s - (h - z)) + (c - z)};
    }
};

// Grid reductions.  Each block reduces its threads' values (warp shuffles, then
// one shuffle tree over the warp totals in warp 0) into part[blockIdx.x*NR + k];
// the last block of the problem (by an atomic ticket) sums all partials in a
// fixed order and returns true with the totals in tot (valid in thread 0).
// Deterministic: the summation tree depends only on the grid shape.
//
// FP32 problems: every product is formed exactly (fmaf split), each thread's
// sum is a compensated float pair, and the block reduces the pairs in
// double-float arithmetic (a value is an unevaluated sum hi + lo of two floats,
// added with Knuth's two-sum; about 44 significant bits) so that the per-pixel
// and per-thread work stays on the FP32 pipe; the block totals and the
// cross-block sum are FP64 (reduce_grid).
__device__ __forceinline__ DF df_add(DF a, DF b) {
    float s = a.hi + b.hi;
    float z = s - a.hi;
    float e = (a.hi - (s - z)) + (b.hi - z);
    e += a.lo + b.lo;
    float h = s + e;
    return DF{h, e - (h - s)};
}

template <typename V> struct RedOps;
template <> struct RedOps<double> {
    __device__ static double zero() { return 0.0; }
    __device__ static double add(double a, double b) { return a + b; }
    __device__ static double shfl(double a, int o) { return __shfl_down_sync(0xffffffffu, a, o); }
    __device__ static void store(double* part, size_t j, double v) { __stcg(part + j, v); }
    __device__ static double load(const double* part, size_t j) { return __ldcg(part + j); }
    __device__ static double total(double v) { return v; }
};
template <> struct RedOps<DF> {
    __device__ static DF zero() { return DF{0.f, 0.f}; }
    __device__ static DF add(DF a, DF b) { return df_add(a, b); }
    __device__ static DF shfl(DF a, int o) {
        return DF{__shfl_down_sync(0xffffffffu, a.hi, o), __shfl_down_sync(0xffffffffu, a.lo, o)};
    }
    __device__ static void store(double* part, size_t j, DF v) {
        __stcg(reinterpret_cast<float2*>(part) + j, make_float2(v.hi, v.lo));
    }
    __device__ static DF load(const double* part, size_t j) {
        float2 y = __ldcg(reinterpret_cast<const float2*>(part) + j);
        return DF{y.x, y.y};
    }
    __device__ static double total(DF v) { return (double)v.hi + (double)v.lo; }
};

// Block reduction in a fixed order: every thread stores its NR values in shared
// memory, then warp w reduces values k = w, w + NW, ... (lane l adds entries
// l, l + 32, ... in order, then a shuffle tree), so that each value costs one
// warp's tree instead of a tree in every warp.  res is valid in thread 0.
template <int NR, int NT, typename V>
__device__ __forceinline__ void block_reduce(const V (&v)[NR], V (&res)[NR]) {
    using O = RedOps<V>;
    constexpr int NW = NT / 32;
    __shared__ V sh[NR][NT];
    __shared__ V shr[NR];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NR; ++k) sh[k][threadIdx.x] = v[k];
    __syncthreads();
    for (int k = warp; k < NR; k += NW) {
        V x = sh[k][lane];
#pragma unroll
        for (int j = 1; j < NW; ++j) x = O::add(x, sh[k][lane + 32 * j]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x = O::add(x, O::shfl(x, o));
        if (lane == 0) shr[k] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NR; ++k) res[k] = shr[k];
    }
}

// The cross-block stage is FP64 for both precisions: each block's total is stored
// as one double (a double-float pair hi + lo converts exactly), and the last block
// sums the partials in double.  Within a block an FP32 problem's values stay
// double-float pairs (FP32 pipe); an FP64 problem's stay doubles.
template <int NR, int NT, typename V>
__device__ __forceinline__ bool reduce_grid(V (&v)[NR], double* part, unsigned* counter, int nblocks,
                                            double (&tot)[NR]) {
    using O = RedOps<V>;
    __shared__ int s_last;
    V bs[NR];
    block_reduce<NR, NT>(v, bs);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NR; ++k) __stcg(part + (size_t)blockIdx.x * NR + k, O::total(bs[k]));
        __threadfence();
        unsigned t = atomicAdd(counter, 1u);
        s_last = (t == (unsigned)(nblocks - 1));
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    // fixed-order FP64 sum of the partials: thread t takes blocks t, t+NT, ... in order
    double x[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        x[k] = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += NT) x[k] += __ldcg(part + (size_t)b * NR + k);
    }
    double tt[NR];
    block_reduce<NR, NT>(x, tt);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NR; ++k) tot[k] = tt[k];
        *counter = 0u;
    }
    return true;
}

// Block + grid reduction of the per-thread accumulators.
template <int NR, int NT, typename T>
__device__ __forceinline__ bool reduce_acc(const Acc<T>* acc, double* part, unsigned* counter, int nblocks,
                                           double (&tot)[NR]) {
    if constexpr (sizeof(T) == 4) {
        DF v[NR];
#pragma unroll
        for (int k = 0; k < NR; ++k) v[k] = acc[k].df();
        return reduce_grid<NR, NT>(v, part, counter, nblocks, tot);
    } else {
        double v[NR];
#pragma unroll
        for (int k = 0; k < NR; ++k) v[k] = acc[k].get();
        return reduce_grid<NR, NT>(v, part, counter, nblocks, tot);
    }
}

// ---------------------------------------------------------------------------
// Pointwise constitutive model (Sec. 2.1).  Strain / stress as (xx, yy, xy)
// with xy the tensor shear component.  Lame constants for plane strain.
template <typename T> __device__ __forceinline__ T rp(T x) { return x > T(0) ? x : T(0); }
template <typename T> __device__ __forceinline__ T rm(T x) { return x < T(0) ? x : T(0); }
template <typename T> __device__ __forceinline__ T hv(T x) { return x > T(0) ? T(1) : T(0); }

// Principal strains e1 >= e2 and the eigen-projector frame of a symmetric
// 2x2 tensor without explicit eigenvectors: with d = (xx-yy)/2, rad =
// sqrt(d^2 + xy^2), u = d/rad, w = xy/rad:
//   P1 = 1/2 [[1+u, w], [w, 1-u]],  P2 = I - P1,  S = [[-w, u], [u, w]]
// (S = n1 n2^T + n2 n1^T).  deg marks coincident principal strains.
// irad = 1/rad when not deg.  FP32 takes rad and 1/rad from one reciprocal
// square root (rsqrtf, 2 ulp) instead of a correctly rounded root and division.
template <typename T>
struct Eig2 {
    T e1, e2, u, w, tr, irad;
    bool deg;
    __device__ __forceinline__ Eig2(T xx, T yy, T xy) {
        tr = xx + yy;
        T d = T(0.5) * (xx - yy);
        T s2 = d * d + xy * xy;
        T rad;
        if constexpr (sizeof(T) == 4) {
            irad = s2 > T(0) ? rsqrtf(s2) : T(0);
            rad = s2 * irad;
        } else {
            rad = sqrt(s2);
            irad = rad > T(0) ? T(1) / rad : T(0);
        }
        e1 = T(0.5) * tr + rad;
        e2 = T(0.5) * tr - rad;
        T scale = fmax(fabs(e1), fabs(e2));
        deg = !(T(2) * rad > T(1e-12) * scale) || rad == T(0);
        if (deg) { u = T(1); w = T(0); }
        else { u = d * irad; w = xy * irad; }
    }
};

// sigma_0^+ (sp) and sigma_0^- (sm) of the strain-spectral split
// (Eq. stress_spectral) and psi_0^+ (Eq. strain_spectral_en).
template <typename T>
__device__ __forceinline__ void spectral_split(T xx, T yy, T xy, T lam, T mu, T* sp, T* sm, T& psip) {
    Eig2<T> g(xx, yy, xy);
    T a1 = rp(g.e1), a2 = rp(g.e2), b1 = rm(g.e1), b2 = rm(g.e2);
    T trp = rp(g.tr), trm = rm(g.tr);
    // eps^+ = a1 P1 + a2 P2
    T hs = T(0.5) * (a1 + a2), hd = T(0.5) * (a1 - a2);
    T epxx = hs + hd * g.u, epyy = hs - hd * g.u, epxy = hd * g.w;
    T ms = T(0.5) * (b1 + b2), md = T(0.5) * (b1 - b2);
    T emxx = ms + md * g.u, emyy = ms - md * g.u, emxy = md * g.w;
    sp[0] = lam * trp + T(2) * mu * epxx;
    sp[1] = lam * trp + T(2) * mu * epyy;
    sp[2] = T(2) * mu * epxy;
    sm[0] = lam * trm + T(2) * mu * emxx;
    sm[1] = lam * trm + T(2) * mu * emyy;
    sm[2] = T(2) * mu * emxy;
    psip = T(0.5) * lam * trp * trp + mu * (a1 * a1 + a2 * a2);
}

template <typename T>
__device__ __forceinline__ T psi_iso(T xx, T yy, T xy, T lam, T mu) {
    T tr = xx + yy;
    return T(0.5) * lam * tr * tr + mu * (xx * xx + yy * yy + T(2) * xy * xy);
}

template <typename T>
__device__ __forceinline__ T psi_spectral(T xx, T yy, T xy, T lam, T mu) {
    Eig2<T> g(xx, yy, xy);
    T a1 = rp(g.e1), a2 = rp(g.e2), trp = rp(g.tr);
    return T(0.5) * lam * trp * trp + mu * (a1 * a1 + a2 * a2);
}

// Volumetric-deviatoric split, Eq. vol_dev_en with the sums over the two in-plane
// components and the 1/3 of the 3-D deviator; K = lambda + 2 mu / 3.
template <typename T>
__device__ __forceinline__ T psi_voldev(T xx, T yy, T xy, T lam, T mu) {
    T tr = xx + yy, K = lam + T(2) * mu / T(3), t3 = tr / T(3);
    T a = xx - t3, b = yy - t3, trp = rp(tr);
    return T(0.5) * K * trp * trp + mu * (a * a + b * b + T(2) * xy * xy);
}

// psi_0^+ of the crack-driving-force model.
template <typename T>
__device__ __forceinline__ T psi_plus(int split, T xx, T yy, T xy, T lam, T mu) {
    const int s = driving_of(split);
    if (s == ISOTROPIC) return psi_iso(xx, yy, xy, lam, mu);
    if (s == VOLDEV) return psi_voldev(xx, yy, xy, lam, mu);
    return psi_spectral(xx, yy, xy, lam, mu);
}

// Stress of the contact model (isotropic for SPECTRAL_STRESSFREE, vol.-dev. for SPECTRAL_VOLDEV).
template <typename T>
__device__ __forceinline__ void stress(int split, T xx, T yy, T xy, T hphi, T lam, T mu, T* s) {
    split = contact_of(split);
    if (split == VOLDEV) {
        // sigma^+ = K <tr>_+ I + 2 mu (eps - 4/9 tr I), sigma^- = K <tr>_- I (exact gradients)
        T tr = xx + yy, K = lam + T(2) * mu / T(3);
        T q = T(4) / T(9) * tr;
        s[0] = hphi * (K * rp(tr) + T(2) * mu * (xx - q)) + K * rm(tr);
        s[1] = hphi * (K * rp(tr) + T(2) * mu * (yy - q)) + K * rm(tr);
        s[2] = hphi * (T(2) * mu * xy);
        return;
    }
    if (split == SPECTRAL) {
        T sp[3], sm[3], psip;
        spectral_split(xx, yy, xy, lam, mu, sp, sm, psip);
        s[0] = hphi * sp[0] + sm[0];
        s[1] = hphi * sp[1] + sm[1];
        s[2] = hphi * sp[2] + sm[2];
    } else {
        T tr = xx + yy;
        s[0] = hphi * (lam * tr + T(2) * mu * xx);
        s[1] = hphi * (lam * tr + T(2) * mu * yy);
        s[2] = hphi * (T(2) * mu * xy);
    }
}

// Energy density psi = h psi_0^+ + psi_0^- of the contact model (Eq. psi_schema).
template <typename T>
__device__ __forceinline__ T energy(int split, T xx, T yy, T xy, T hphi, T lam, T mu) {
    split = contact_of(split);
    if (split == VOLDEV) {
        T tr = xx + yy, K = lam + T(2) * mu / T(3), trm = rm(tr);
        return hphi * psi_voldev(xx, yy, xy, lam, mu) + T(0.5) * K * trm * trm;
    }
    if (split == SPECTRAL) {
        Eig2<T> g(xx, yy, xy);
        T a1 = rp(g.e1), a2 = rp(g.e2), b1 = rm(g.e1), b2 = rm(g.e2);
        T trp = rp(g.tr), trm = rm(g.tr);
        T pp = T(0.5) * lam * trp * trp + mu * (a1 * a1 + a2 * a2);
        T pm = T(0.5) * lam * trm * trm + mu * (b1 * b1 + b2 * b2);
        return hphi * pp + pm;
    }
    return hphi * psi_iso(xx, yy, xy, lam, mu);
}

// Tangent C:p of the contact model at strain eps (Sec. 3.1.1).  Spectral:
// Daleckii-Krein derivative of eps -> eps^+ in the frame (P1, P2, S):
//   D+[p] = H(e1)(P1:p)P1 + H(e2)(P2:p)P2 + g12 (S:p/2) S,
//   g12 = (<e1>_+ - <e2>_+)/(e1 - e2)  (H(e1) for coincident e1 = e2),
// sigma' = h (lam H(tr) tr p I + 2 mu D+) + lam (1 - H(tr)) tr p I + 2 mu (p - D+).
template <typename T>
__device__ __forceinline__ void tangent(int split, T xx, T yy, T xy, T hphi, T lam, T mu,
                                        T pxx, T pyy, T pxy, T* out) {
    T trp = pxx + pyy;
    split = contact_of(split);
    if (split == VOLDEV) {
        T K = lam + T(2) * mu / T(3), Ht = hv(xx + yy);
        T q = T(4) / T(9) * trp;
        out[0] = hphi * (K * Ht * trp + T(2) * mu * (pxx - q)) + K * (T(1) - Ht) * trp;
        out[1] = hphi * (K * Ht * trp + T(2) * mu * (pyy - q)) + K * (T(1) - Ht) * trp;
        out[2] = hphi * (T(2) * mu * pxy);
        return;
    }
    if (split == SPECTRAL) {
        Eig2<T> g(xx, yy, xy);
        T dxx, dyy, dxy;
        if (g.deg) {
            T H = hv(g.e1);
            dxx = H * pxx; dyy = H * pyy; dxy = H * pxy;
        } else {
            T H1 = hv(g.e1), H2 = hv(g.e2);
            // divided difference (<e1>_+ - <e2>_+)/(e1 - e2): H(e1) when e1 and e2 have
            // the same sign (exactly, as the quotient of equal values), e1 / (2 rad)
            // when they straddle zero (no cancellation there); FP32 avoids the division
            T g12;
            if constexpr (sizeof(T) == 4) g12 = (g.e1 > T(0) && g.e2 < T(0)) ? g.e1 * (T(0.5) * g.irad) : H1;
            else g12 = (rp(g.e1) - rp(g.e2)) / (g.e1 - g.e2);
            T u = g.u, w = g.w;
            T P1p = T(0.5) * ((T(1) + u) * pxx + (T(1) - u) * pyy + T(2) * w * pxy);
            T P2p = T(0.5) * ((T(1) - u) * pxx + (T(1) + u) * pyy - T(2) * w * pxy);
            T Sp = T(0.5) * (-w * pxx + w * pyy + T(2) * u * pxy);
            T c1 = H1 * P1p, c2 = H2 * P2p, c3 = g12 * Sp;
            dxx = T(0.5) * (c1 * (T(1) + u) + c2 * (T(1) - u)) - c3 * w;
            dyy = T(0.5) * (c1 * (T(1) - u) + c2 * (T(1) + u)) + c3 * w;
            dxy = T(0.5) * (c1 * w - c2 * w) + c3 * u;
        }
        T Ht = hv(g.tr);
        T lp = lam * Ht * trp, lm = lam * (T(1) - Ht) * trp;
        out[0] = hphi * (lp + T(2) * mu * dxx) + lm + T(2) * mu * (pxx - dxx);
        out[1] = hphi * (lp + T(2) * mu * dyy) + lm + T(2) * mu * (pyy - dyy);
        out[2] = hphi * (T(2) * mu * dxy) + T(2) * mu * (pxy - dxy);
    } else {
        out[0] = hphi * (lam * trp + T(2) * mu * pxx);
        out[1] = hphi * (lam * trp + T(2) * mu * pyy);
        out[2] = hphi * (T(2) * mu * pxy);
    }
}

}  // namespace pff
