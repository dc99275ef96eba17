// ops.cuh -- per-pixel prologues / epilogues / finalizers of the load step.
//
// Mechanics (Sec. 3.1.1), one operator application per CG iteration:
//   K1 row_fwd  FCgIn     : p = r + b p (previous iteration's b); tau = C_m : p; p.tau -> a;
//                           FFT rows
//   K2 col      FColGamma : Gamma projection between column FFTs
//   K3 row_inv  FCgOut    : q = A p; x += a p, r -= a q; explicit r.r -> stop test, b
// Newton residual (Eq. elasticity_nodal): FNewtonIn / FColGammaN / FNewtonOut.
// Phase field (Algorithm 1), two operator applications per BCCG iteration:
//   A1 FPfA1 (p = -r + b p, masked) -> A2 lap -> A3 FPfA3 (p.Jp, r.p -> alpha)
//   B1 FPfB1 (v = max(v + alpha p, v_con)) -> B2 lap -> B3 FPfB3 (r = Jv - b, active set,
//   r.r, r.r_old -> beta, convergence).
// Flags: see Ctrl in common.cuh.
#pragma once
#include "common.cuh"
#include "fft.cuh"

namespace pff {

constexpr int PF_STALL = 64;    // FP32 BCCG: iterations without a new smallest ||r|| that end a solve

// Lame constants per unit E in the storage type, read once per block (a per-pixel
// double-to-float conversion would run on the narrow FP64 pipe).
template <typename T>
struct LameC {
    T lc, mc;
    LameC() = default;
    __device__ __forceinline__ explicit LameC(const Desc<T>& d) : lc(T(d.k.lam_c)), mc(T(d.k.mu_c)) {}
    __device__ __forceinline__ void at(const Desc<T>& d, size_t i, T& lam, T& mu) const {
        T E = d.E[i];
        lam = lc * E;
        mu = mc * E;
    }
};
template <typename T>
__device__ __forceinline__ void lame_at(const Desc<T>& d, size_t i, T& lam, T& mu) {
    T E = d.E[i];
    lam = T(d.k.lam_c) * E;
    mu = T(d.k.mu_c) * E;
}

// FP64 sign of a*x - kappa*l - b from FP32 operands; kept out of line so that it
// only runs for the rare residuals within FP32 rounding of zero.
static __device__ __noinline__ bool resid_positive_fp64(float a, float x, double kappa, float l, float b) {
    return ((double)a * (double)x - kappa * (double)l - (double)b) > 0.0;
}
// FP64 sign of the recurrence residual R + alpha J p from the FP32 stored R and J p
// and the FP64 step length (out of line for the same reason).
static __device__ __noinline__ bool recur_positive_fp64(float R, double alpha, float Jp) {
    return fma(alpha, (double)Jp, (double)R) > 0.0;
}
template <typename T> __device__ __forceinline__ T hdeg(T phi) { return (T(1) - phi) * (T(1) - phi); }

// weighted (Frobenius) inner product of symmetric tensors stored (xx, yy, xy)
template <typename T>
__device__ __forceinline__ void wdot(Acc<T>& a, T x0, T x1, T x2, T y0, T y1, T y2) {
    a.addp(x0, y0);
    a.addp(x1, y1);
    a.addp(x2 + x2, y2);
}

struct NoCtx {};

// ---------------------------------------------------------------- mechanics
template <typename T>
struct FNewtonIn {   // eps* += theta (rounds > 0), sigma(eps_bar + eps*, phi)
    static constexpr int NR = 0;
    struct Ctx { T eb[3]; int fold; int split; LameC<T> lm; };
    __device__ static bool skip(const Desc<T>& d) { return ldflag(&d.ctrl->nd_a); }
    __device__ static Ctx prep(const Desc<T>& d) {
        Ctx c{{}, 0, 0, LameC<T>(d)};
        for (int k = 0; k < 3; ++k) c.eb[k] = T(ldd(&d.ctrl->eps_bar[k]));
        c.fold = ldflag(&d.ctrl->newton_it) > 0;
        c.split = d.k.split;
        return c;
    }
    __device__ static void pixel(const Desc<T>& d, const Ctx& c, size_t i, T (&v)[3], Acc<T>*) {
        T e0 = d.eps[0][i], e1 = d.eps[1][i], e2 = d.eps[2][i];
        if (c.fold) {
            e0 += d.th[0][i]; e1 += d.th[1][i]; e2 += d.th[2][i];
            d.eps[0][i] = e0; d.eps[1][i] = e1; d.eps[2][i] = e2;
        }
        T lam, mu;
        c.lm.at(d, i, lam, mu);
        stress(c.split, c.eb[0] + e0, c.eb[1] + e1, c.eb[2] + e2, hdeg(d.phi[i]), lam, mu, v);
    }
    __device__ static void finalize(const Desc<T>&, const double*) {}
};

struct FColGammaN {   // Newton trio column pass: copies nd_b = nd_a
    template <typename T> __device__ static bool skip(const Desc<T>& d) {
        int f = ldflag(&d.ctrl->nd_a);
        if (blockIdx.x == 0 && threadIdx.x == 0) d.ctrl->nd_b = f;
        return f;
    }
    template <typename T> __device__ static void apply(const ModeK<T>& m, int kx, int ky, typename CT<T>::t (&v)[3]) {
        gamma_apply(m, kx, ky, v);
    }
};

template <typename T>
struct FNewtonOut {   // R = P sigma; CG start r = p = -R, theta = 0; Newton test
    static constexpr int NR = 1;
    using Ctx = NoCtx;
    __device__ static bool skip(const Desc<T>& d) { return ldflag(&d.ctrl->nd_b); }
    __device__ static Ctx prep(const Desc<T>&) { return Ctx{}; }
    __device__ static void pixel(const Desc<T>& d, const Ctx&, size_t i, T (&v)[3], Acc<T>* acc) {
        wdot(acc[0], v[0], v[1], v[2], v[0], v[1], v[2]);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            d.r[k][i] = -v[k];
            d.p[k][i] = -v[k];
            d.th[k][i] = T(0);
        }
    }
    __device__ static void finalize(const Desc<T>& d, const double* tot) {
        Ctrl* c = d.ctrl;
        const Consts& k = d.k;
        double R2 = tot[0], rn = sqrt(R2);
        // ||C_0(E) : eps_bar|| = sqrt(sum E^2) * |C_0(1) : eps_bar|
        double eb0 = c->eps_bar[0], eb1 = c->eps_bar[1], eb2 = c->eps_bar[2];
        double tr = eb0 + eb1;
        double s0 = k.lam_c * tr + 2.0 * k.mu_c * eb0, s1 = k.lam_c * tr + 2.0 * k.mu_c * eb1, s2 = 2.0 * k.mu_c * eb2;
        double target = k.mech_tol * sqrt(c->sumE2) * sqrt(s0 * s0 + s1 * s1 + 2.0 * s2 * s2);
        c->mech_target = target;
        c->R2 = R2;
        if (rn <= target || c->newton_it >= k.max_newton) {
            if (rn > target) c->status |= 1;
            c->nd_a = 1;
            c->cg_a = 1;
            c->cg_b = 1;
        } else {
            const bool linear = (contact_of(k.split) == ISOTROPIC);
            c->cg_target = linear ? target : fmax(target, k.mech_cg_rtol * rn);
            c->rr = R2;
            c->cg_it = 0;
            c->cg_break = 0;
            c->cg_a = 0;
            c->cg_b = 0;
            c->newton_it += 1;
            if (linear) {   // a linear model takes one Newton step (Sec. 3.1.1)
                c->nd_a = 1;
                c->needs_fold = 1;
            }
        }
    }
};

// CG iteration k, split over the operator's two row passes (Sec. 3.1.1; the CG of
// Eq. elasticity_newton_linear):
//   FCgIn  (row forward): p_k = r_k + beta_{k-1} p_{k-1} (k > 0), tau = C_m : p_k, the
//          real FFT of tau along x; p_k.tau -> alpha_k = r_k.r_k / p_k.A p_k, where
//          p.Ap = p.P tau = p.tau because every iterate lies in range(P) (P = F^-1 Gamma F,
//          an orthogonal projection).
//   FCgOut (row inverse): q = A p_k; theta += alpha p_k, r_{k+1} = r_k - alpha q; the
//          explicit r_{k+1}.r_{k+1} -> stopping test and beta_k = r_{k+1}.r_{k+1} / r_k.r_k.
// q is never stored.  Flags: FCgIn skips on cg_b (set by the previous FCgOut's stopping
// test) and copies it to cg_a, which the column pass and FCgOut read.
template <typename T>
struct FCgIn {
    static constexpr int NR = 1;
    struct Ctx { T beta; int upd; int iso; T eb[3]; int split; LameC<T> lm; };
    __device__ static bool skip(const Desc<T>& d) {
        int f = ldflag(&d.ctrl->cg_b);
        if (blockIdx.x == 0 && threadIdx.x == 0) d.ctrl->cg_a = f;
        return f;
    }
    __device__ static Ctx prep(const Desc<T>& d) {
        Ctx c{T(0), 0, 0, {}, 0, LameC<T>(d)};
        c.upd = ldflag(&d.ctrl->cg_it) > 0;
        c.beta = T(ldd(&d.ctrl->beta));
        for (int k = 0; k < 3; ++k) c.eb[k] = T(ldd(&d.ctrl->eps_bar[k]));
        c.split = d.k.split;
        c.iso = contact_of(d.k.split) == ISOTROPIC;   // the isotropic tangent does not depend on eps
        return c;
    }
    // two-phase pixel: all loads of a thread's pixels are issued before any store
    struct In { T p[3], r[3], e[3], phi, E; };
    __device__ static In load(const Desc<T>& d, const Ctx& c, size_t i) {
        In a;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            a.p[k] = d.p[k][i];
            if (c.upd) a.r[k] = d.r[k][i];
            a.e[k] = c.iso ? T(0) : d.eps[k][i];
        }
        a.phi = d.phi[i];
        a.E = d.E[i];
        return a;
    }
    __device__ static void pixel(const Desc<T>& d, const Ctx& c, size_t i, const In& a, T (&v)[3], Acc<T>* acc) {
        T p[3];
        if (c.upd) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                p[k] = a.r[k] + c.beta * a.p[k];
                d.p[k][i] = p[k];
            }
        } else {
#pragma unroll
            for (int k = 0; k < 3; ++k) p[k] = a.p[k];
        }
        T lam = c.lm.lc * a.E, mu = c.lm.mc * a.E;
        tangent(c.split, c.eb[0] + a.e[0], c.eb[1] + a.e[1], c.eb[2] + a.e[2], hdeg(a.phi), lam, mu,
                p[0], p[1], p[2], v);
        wdot(acc[0], p[0], p[1], p[2], v[0], v[1], v[2]);
    }
    __device__ static void finalize(const Desc<T>& d, const double* tot) {
        Ctrl* c = d.ctrl;
        const double pAp = tot[0];
        c->pAp = pAp;
        if (!(pAp > 0.0)) {   // p.Ap <= 0: stop (A8); every block has read cg_b already
            c->cg_break = 1;
            c->alpha = 0.0;
            c->cg_a = 1;
            c->cg_b = 1;
        } else {
            c->alpha = c->rr / pAp;
        }
    }
};

struct FColGammaCG {   // CG column pass (skips with cg_a)
    template <typename T> __device__ static bool skip(const Desc<T>& d) { return ldflag(&d.ctrl->cg_a); }
    template <typename T> __device__ static void apply(const ModeK<T>& m, int kx, int ky, typename CT<T>::t (&v)[3]) {
        gamma_apply(m, kx, ky, v);
    }
};

template <typename T>
struct FCgOut {
    static constexpr int NR = 1;
    struct Ctx { T alpha; };
    __device__ static bool skip(const Desc<T>& d) { return ldflag(&d.ctrl->cg_a); }
    __device__ static Ctx prep(const Desc<T>& d) { return Ctx{T(ldd(&d.ctrl->alpha))}; }
    struct In { T th[3], r[3], p[3]; };
    __device__ static In load(const Desc<T>& d, const Ctx&, size_t i) {
        In a;
#pragma unroll
        for (int k = 0; k < 3; ++k) { a.th[k] = d.th[k][i]; a.r[k] = d.r[k][i]; a.p[k] = d.p[k][i]; }
        return a;
    }
    __device__ static void pixel(const Desc<T>& d, const Ctx& c, size_t i, const In& a, T (&v)[3], Acc<T>* acc) {
        T r[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            d.th[k][i] = a.th[k] + c.alpha * a.p[k];
            r[k] = a.r[k] - c.alpha * v[k];
            d.r[k][i] = r[k];
        }
        wdot(acc[0], r[0], r[1], r[2], r[0], r[1], r[2]);
    }
    __device__ static void finalize(const Desc<T>& d, const double* tot) {
        Ctrl* c = d.ctrl;
        const double rr = tot[0], rr_old = c->rr;
        c->cg_it += 1;
        c->cg_total += 1;
        c->beta = rr_old > 0.0 ? rr / rr_old : 0.0;
        c->rr = rr;
        const bool conv = sqrt(rr) <= c->cg_target;
        if (conv || c->cg_it >= d.k.max_cg) {
            if (!conv) c->status |= 1;
            c->cg_b = 1;
        } else {
            c->cg_b = 0;
        }
    }
};

// elementwise: eps* += theta after a linear model's single Newton step
template <typename T>
struct FFold {
    static constexpr int NR = 0;
    using Ctx = NoCtx;
    __device__ static bool skip(const Desc<T>& d) { return !ldflag(&d.ctrl->needs_fold); }
    __device__ static Ctx prep(const Desc<T>&) { return Ctx{}; }
    __device__ static void pixel(const Desc<T>& d, const Ctx&, size_t i, Acc<T>*) {
        d.eps[0][i] += d.th[0][i];
        d.eps[1][i] += d.th[1][i];
        d.eps[2][i] += d.th[2][i];
    }
    __device__ static void finalize(const Desc<T>&, const double*) {}
};

// ---------------------------------------------------------------- scalar-field transforms
template <typename T>
struct FPhiIn {   // input phi (driving force and energy trios)
    static constexpr int NR = 0;
    using Ctx = NoCtx;
    __device__ static bool skip(const Desc<T>&) { return false; }
    __device__ static Ctx prep(const Desc<T>&) { return Ctx{}; }
    __device__ static void pixel(const Desc<T>& d, const Ctx&, size_t i, T (&v)[1], Acc<T>*) { v[0] = d.phi[i]; }
    __device__ static void finalize(const Desc<T>&, const double*) {}
};

struct FColLapDF {   // column pass of the step's lap(phi); clears needs_fold (read by the fold kernel before)
    template <typename T> __device__ static bool skip(const Desc<T>& d) {
        if (blockIdx.x == 0 && threadIdx.x == 0) d.ctrl->needs_fold = 0;
        return false;
    }
    template <typename T> __device__ static void apply(const ModeK<T>& m, int kx, int ky, typename CT<T>::t (&v)[1]) {
        lap_apply(m, kx, ky, v);
    }
};

struct FColLapPlain {
    template <typename T> __device__ static bool skip(const Desc<T>&) { return false; }
    template <typename T> __device__ static void apply(const ModeK<T>& m, int kx, int ky, typename CT<T>::t (&v)[1]) {
        lap_apply(m, kx, ky, v);
    }
};

// Low-pass filter of the microstructure generator (Sec. 3.3): keeps the modes
// with 0 < |q| <= 2 pi / L_cut, decided as kx^2 (Ly L_cut)^2 + ky^2 (Lx L_cut)^2
// <= (Lx Ly)^2 with unfused FP64 products and sum.
struct FColLowPass {
    template <typename T> __device__ static bool skip(const Desc<T>&) { return false; }
    template <typename T> __device__ static void apply(const ModeK<T>& m, int kx, int ky, typename CT<T>::t (&v)[1]) {
        const int sk = signed_k(ky, m.ny);
        const double lhs = __dadd_rn(__dmul_rn((double)kx * (double)kx, m.kc->lp_a),
                                     __dmul_rn((double)sk * (double)sk, m.kc->lp_b));
        const bool keep = (kx != 0 || sk != 0) && lhs <= m.kc->lp_c;
        const T f = keep ? m.inv_n : T(0);
        v[0].x *= f;
        v[0].y *= f;
    }
};

struct FColGammaPlain {
    template <typename T> __device__ static bool skip(const Desc<T>&) { return false; }
    template <typename T> __device__ static void apply(const ModeK<T>& m, int kx, int ky, typename CT<T>::t (&v)[3]) {
        gamma_apply(m, kx, ky, v);
    }
};

template <typename T>
struct FLapOut {   // lap = nabla^2_N phi
    static constexpr int NR = 0;
    using Ctx = NoCtx;
    __device__ static bool skip(const Desc<T>&) { return false; }
    __device__ static Ctx prep(const Desc<T>&) { return Ctx{}; }
    __device__ static void pixel(const Desc<T>& d, const Ctx&, size_t i, T (&v)[1], Acc<T>*) { d.lap[i] = v[0]; }
    __device__ static void finalize(const Desc<T>&, const double*) {}
};

template <typename T>
struct FEnergyOut {   // F_f = c sum (f(phi) - ell^2 phi lap phi) dA (Eq. Ff with Parseval)
    static constexpr int NR = 1;
    using Ctx = NoCtx;
    __device__ static bool skip(const Desc<T>&) { return false; }
    __device__ static Ctx prep(const Desc<T>&) { return Ctx{}; }
    __device__ static void pixel(const Desc<T>& d, const Ctx&, size_t i, T (&v)[1], Acc<T>* acc) {
        T ph = d.phi[i];
        T f = d.k.fracture == AT1 ? ph : ph * ph;
        acc[0].add(f);
        acc[0].addp(-T(d.k.ell2) * ph, v[0]);
    }
    __device__ static void finalize(const Desc<T>& d, const double* tot) {
        d.ctrl->Ff = d.k.c * tot[0] * d.k.dA;
    }
};

// copies for the operator entry points: input r[], output q[]
template <typename T, int NC>
struct FCopyIn {
    static constexpr int NR = 0;
    using Ctx = NoCtx;
    __device__ static bool skip(const Desc<T>&) { return false; }
    __device__ static Ctx prep(const Desc<T>&) { return Ctx{}; }
    __device__ static void pixel(const Desc<T>& d, const Ctx&, size_t i, T (&v)[NC], Acc<T>*) {
#pragma unroll
        for (int k = 0; k < NC; ++k) v[k] = d.r[k][i];
    }
    __device__ static void finalize(const Desc<T>&, const double*) {}
};
template <typename T, int NC>
struct FCopyOut {
    static constexpr int NR = 0;
    using Ctx = NoCtx;
    __device__ static bool skip(const Desc<T>&) { return false; }
    __device__ static Ctx prep(const Desc<T>&) { return Ctx{}; }
    __device__ static void pixel(const Desc<T>& d, const Ctx&, size_t i, T (&v)[NC], Acc<T>*) {
#pragma unroll
        for (int k = 0; k < NC; ++k) d.q[k][i] = v[k];
    }
    __device__ static void finalize(const Desc<T>&, const double*) {}
};

// ---------------------------------------------------------------- phase field
// BCCG start (Algorithm 1 lines 1-5) after the rescale of lines 4-10 of Algorithm 4:
// eps <- gamma eps; a = eta/dt + 2 psi_0^+ + c f''; b = -F_phi(phi_n);
// v_con = phi_con(phi_n) - phi_n <= 0; v^0 = 0; r^0 = -b masked; p^0 = -r^0.
template <typename T>
struct FPfInit {
    static constexpr int NR = 4;
    struct Ctx { double g; int resc; double eb[3]; double eta_dt; int frozen; };
    __device__ static bool skip(const Desc<T>&) { return false; }
    __device__ static Ctx prep(const Desc<T>& d) {
        Ctx c;
        c.g = ldd(&d.ctrl->gamma);
        c.resc = ldflag(&d.ctrl->rescaled);
        for (int k = 0; k < 3; ++k) c.eb[k] = c.g * ldd(&d.ctrl->eps_bar[k]);
        c.eta_dt = ldflag(&d.ctrl->use_override) ? ldd(&d.ctrl->eta_dt_override) : d.k.eta_dt;
        c.frozen = ldflag(&d.ctrl->con_frozen);
        return c;
    }
    __device__ static void pixel(const Desc<T>& d, const Ctx& c, size_t i, Acc<T>* acc) {
        const Consts& k = d.k;
        T e0 = d.eps[0][i], e1 = d.eps[1][i], e2 = d.eps[2][i];
        if (c.resc) {
            T g = T(c.g);
            e0 *= g; e1 *= g; e2 *= g;
            d.eps[0][i] = e0; d.eps[1][i] = e1; d.eps[2][i] = e2;
        }
        double E = (double)d.E[i];
        double lam = k.lam_c * E, mu = k.mu_c * E;
        double psi = psi_plus<double>(k.split, c.eb[0] + (double)e0, c.eb[1] + (double)e1, c.eb[2] + (double)e2, lam, mu);
        T ph = d.phi[i];
        double phd = (double)ph;
        double fp = k.fracture == AT1 ? 1.0 : 2.0 * phd;
        T a = T(c.eta_dt + 2.0 * psi + k.cf2);
        T b = T(2.0 * (1.0 - phd) * psi - k.c * fp + k.kappa * (double)d.lap[i]);
        T pcon = c.frozen ? d.aux[i] : ((k.irrev == CRACK_SET) ? (ph >= T(k.crack_thr) ? ph : T(0)) : ph);
        T vcon = pcon - ph;
        T v = T(0) < vcon ? vcon : T(0);
        bool at = (v == vcon);
        T r = -b;
        d.lap[i] = r;                 // unmasked residual R = J v - b (v = 0)
        bool active = at && (r > T(0));
        if (active) r = T(0);
        d.th[0][i] = v;
        d.th[1][i] = r;
        d.th[2][i] = -r;
        d.r[0][i] = a;
        d.r[1][i] = b;
        d.r[2][i] = vcon;
        d.flags[i] = (uint8_t)((at ? 1 : 0) | (active ? 2 : 0));
        acc[0].addp(r, r);
        acc[1].addp(b, b);
        acc[2].add(a);
        acc[3].addp(a * r, r);   // sum a p^2 of the first direction p = -r
    }
    __device__ static void finalize(const Desc<T>& d, const double* tot) {
        Ctrl* c = d.ctrl;
        const Consts& k = d.k;
        double rn = sqrt(tot[0]);
        double target = fmax(fmax(k.pf_tol * rn, k.pf_atol), k.pf_floor * sqrt(tot[1]));
        c->pf_rr = tot[0];
        c->pf_target = target;
        c->pf_it = 0;
        c->pf_break = 0;
        c->n_active = 0;
        c->pf_full = 1;
        c->pf_force = 0;
        c->pf_confirm = 0;
        c->pf_since_full = 0;
        c->pf_full_iters = 0;
        c->pf_rsel = 0;
        c->pf_abar = tot[2] * k.inv_n;
        c->pf_rz = 0.0;
        c->pf_pap = tot[3];
        c->pf_rp = -tot[0];
        c->bar_count = 0;
        c->bar_abort = 0;
        c->pf_last_full = rn;
        c->pf_best = rn;
        c->pf_best_it = 0;
        int done = rn <= target;
        c->pf_a = done;
        c->pf_b = done;
        if (c->rescaled)
            for (int j = 0; j < 3; ++j) c->eps_bar[j] *= c->gamma;
    }
};

// The BCCG residual r is double-buffered: the fused iterate kernel writes the
// recurrence residual beside the previous one, which an explicit evaluation in
// the same iteration still needs for beta.
template <typename T> __device__ __forceinline__ T* pf_r(const Desc<T>& d, int sel) { return sel ? d.q[1] : d.th[1]; }

template <typename T>
struct FPfA1 {   // p = -r + beta p (Algorithm 1) or p = -z + beta p (preconditioned), zero on the active set; input p
    static constexpr int NR = 0;
    struct Ctx { T beta; int upd; int pre; const T* r; };
    __device__ static bool skip(const Desc<T>& d) {
        if (d.k.pf_precond) return ldflag(&d.ctrl->pf_a);   // copied by the preconditioner's first pass
        int f = ldflag(&d.ctrl->pf_b);
        if (blockIdx.x == 0 && threadIdx.x == 0) d.ctrl->pf_a = f;
        return f;
    }
    __device__ static Ctx prep(const Desc<T>& d) {
        Ctx c;
        c.pre = d.k.pf_precond;
        c.upd = c.pre || ldflag(&d.ctrl->pf_it) > 0;
        c.beta = T(ldd(&d.ctrl->pf_beta));
        c.r = c.pre ? d.q[2] : pf_r(d, ldflag(&d.ctrl->pf_rsel));   // z or r
        return c;
    }
    struct In { T p, r; uint8_t fl; };
    __device__ static In load(const Desc<T>& d, const Ctx& c, size_t i) {
        In a{d.th[2][i], T(0), 0};
        if (c.upd) { a.r = c.r[i]; a.fl = d.flags[i]; }
        return a;
    }
    __device__ static void pixel(const Desc<T>& d, const Ctx& c, size_t i, const In& a, T (&v)[1], Acc<T>*) {
        T p = a.p;
        if (c.upd) {
            p = -a.r + c.beta * p;
            if (a.fl & 2) p = T(0);
            d.th[2][i] = p;
        }
        v[0] = p;
    }
    __device__ static void finalize(const Desc<T>&, const double*) {}
};

// Preconditioned variant (pff_params.pf_precondition): z = M^-1 r on the free set
// with M = a_mean - 2 c ell^2 nabla^2_N, i.e. (a_mean + 2 c ell^2 |2 pi q|^2)^-1 per
// Fourier mode -- the constant-coefficient part of J, inverted exactly by one FFT
// pair.  Three passes: the residual forward along x, the mode multiplier along y,
// the inverse along x with the masking and r.z, r_old.z -> beta (Polak-Ribiere in
// the preconditioned inner product, r_old.z_old = -r_old.p_old after the step).
template <typename T>
struct FPfZIn {   // input r; first pass of an iteration: copies the stop flag
    static constexpr int NR = 0;
    struct Ctx { const T* r; };
    __device__ static bool skip(const Desc<T>& d) {
        int f = ldflag(&d.ctrl->pf_b);
        if (blockIdx.x == 0 && threadIdx.x == 0) d.ctrl->pf_a = f;
        return f;
    }
    __device__ static Ctx prep(const Desc<T>& d) { return Ctx{pf_r(d, ldflag(&d.ctrl->pf_rsel))}; }
    struct In { T r; };
    __device__ static In load(const Desc<T>&, const Ctx& c, size_t i) { return In{c.r[i]}; }
    __device__ static void pixel(const Desc<T>&, const Ctx&, size_t, const In& a, T (&v)[1], Acc<T>*) { v[0] = a.r; }
    __device__ static void finalize(const Desc<T>&, const double*) {}
};

struct FColPrecond {
    template <typename T> __device__ static bool skip(const Desc<T>& d) { return ldflag(&d.ctrl->pf_a); }
    template <typename T> __device__ static void mode_prep(const Desc<T>& d, ModeK<T>& m) {
        const double ab = ldd(&d.ctrl->pf_abar);
        // a_mean >= eta/dt > 0 in Algorithm 4; a zero mean (eta/dt = 0 and no load) falls
        // back to the smallest nonzero Laplacian eigenvalue scale
        m.pre_a = T(ab > 0.0 ? ab : d.k.kappa * d.k.two_pi_over_Lx * d.k.two_pi_over_Lx);
        m.pre_k = T(d.k.kappa);
    }
    template <typename T> __device__ static void apply(const ModeK<T>& m, int kx, int ky, typename CT<T>::t (&v)[1]) {
        T qx = T(kx) * m.cx;
        T qy = T(signed_k(ky, m.ny)) * m.cy;
        T f = m.inv_n / (m.pre_a + m.pre_k * (qx * qx + qy * qy));
        v[0].x *= f;
        v[0].y *= f;
    }
};

template <typename T>
struct FPfZOut {   // z = M^-1 r masked to the free set (into q[2]); r.z, r_old.z -> beta
    static constexpr int NR = 2;
    struct Ctx { const T* r; const T* ro; };
    __device__ static bool skip(const Desc<T>& d) { return ldflag(&d.ctrl->pf_a); }
    __device__ static Ctx prep(const Desc<T>& d) {
        const int sel = ldflag(&d.ctrl->pf_rsel);
        return Ctx{pf_r(d, sel), pf_r(d, sel ^ 1)};
    }
    struct In { T r, ro; uint8_t fl; };
    __device__ static In load(const Desc<T>& d, const Ctx& c, size_t i) { return In{c.r[i], c.ro[i], d.flags[i]}; }
    __device__ static void pixel(const Desc<T>& d, const Ctx&, size_t i, const In& a, T (&v)[1], Acc<T>* acc) {
        const T z = (a.fl & 2) ? T(0) : v[0];
        d.q[2][i] = z;
        acc[0].addp(z, a.r);
        acc[1].addp(z, a.ro);
    }
    __device__ static void finalize(const Desc<T>& d, const double* tot) {
        Ctrl* c = d.ctrl;
        const double den = c->pf_rz;
        // the first iteration has no previous residual (beta = 0, p = -z)
        c->pf_beta = (c->pf_it > 0 && den != 0.0) ? (tot[0] - tot[1]) / den : 0.0;
        c->pf_rz = tot[0];
    }
};

struct FColLapPF {
    template <typename T> __device__ static bool skip(const Desc<T>& d) { return ldflag(&d.ctrl->pf_a); }
    template <typename T> __device__ static void apply(const ModeK<T>& m, int kx, int ky, typename CT<T>::t (&v)[1]) {
        lap_apply(m, kx, ky, v);
    }
};

template <typename T>
struct FPfA3 {   // J p; p.Jp, r.p -> alpha = -(r.p)/(p.Jp)
    static constexpr int NR = 2;
    struct Ctx { T kappa; const T* r; };
    __device__ static bool skip(const Desc<T>& d) { return ldflag(&d.ctrl->pf_a); }
    __device__ static Ctx prep(const Desc<T>& d) { return Ctx{T(d.k.kappa), pf_r(d, ldflag(&d.ctrl->pf_rsel))}; }
    struct In { T p, a, r; };
    __device__ static In load(const Desc<T>& d, const Ctx& c, size_t i) { return In{d.th[2][i], d.r[0][i], c.r[i]}; }
    __device__ static void pixel(const Desc<T>& d, const Ctx& c, size_t i, const In& a, T (&v)[1], Acc<T>* acc) {
        T Jp = a.a * a.p - c.kappa * v[0];
        d.q[0][i] = Jp;
        acc[0].addp(a.p, Jp);
        acc[1].addp(a.r, a.p);
    }
    __device__ static void finalize(const Desc<T>& d, const double* tot) {
        Ctrl* c = d.ctrl;
        c->pJp = tot[0];
        c->pf_rp = tot[1];
        if (!(tot[0] > 0.0)) {
            c->pf_break = 1;
            c->pf_alpha = 0.0;
        } else {
            c->pf_alpha = -tot[1] / tot[0];
        }
    }
};

// ---- Algorithm 1 iteration in three operator passes (the default, unpreconditioned path)
// p.Jp = sum a p^2 - kappa sum p lap_N p, and -sum p lap_N p = (1/(nx ny)) sum_k |2 pi q|^2
// |p^_k|^2 over the full spectrum (Parseval), so alpha = -(r.p)/(p.Jp) is known after the
// column pass, and the row-inverse pass that forms J p applies the iterate at once:
//   FPfA1      (row forward): p = -r + beta p, zero on the active set
//   FColLapPFQ (column)     : sum over the modes of w(kx) |2 pi q|^2 |p^|^2 (w = 2 on the kx
//                             columns that stand for two modes, else 1); alpha
//   FPfA3B     (row inverse): J p = a p - kappa lap_N p; v = max(v + alpha p, v_con); the
//                             residual recurrence R + alpha J p; active set; r' and its dots
// sum a p^2 and r.p of the next direction p' = -r' + beta p (free pixels; 0 on the active set)
// come from sums of the iteration that forms r': sum a p'^2 = S1 - 2 beta S2 + beta^2 S3 and
// r'.p' = -r'.r' + beta S4 with S1 = sum a r'^2, S2 = sum a r' p, S3 = sum a p^2 (free
// pixels) and S4 = r'.p (pf_next_dir); the first direction p = -r from the start's sums.
// (The preconditioned variant and the persistent kernel keep FPfA1 / FColLapPF / FPfA3 / FPfB1.)
struct FColLapPFQ {
    static constexpr int NR = 1;
    template <typename T> __device__ static bool skip(const Desc<T>& d) { return ldflag(&d.ctrl->pf_a); }
    template <typename T>
    __device__ static void accum(const ModeK<T>& m, int kx, int ky, const typename CT<T>::t (&v)[1], Acc<T>* acc) {
        if (2 * kx > m.nx) return;   // padding columns of the spectrum rows hold no modes
        const T qx = T(kx) * m.cx, qy = T(signed_k(ky, m.ny)) * m.cy;
        const T w = (kx == 0 || 2 * kx == m.nx) ? T(1) : T(2);
        const T q2 = w * (qx * qx + qy * qy);
        acc[0].addp(q2 * v[0].x, v[0].x);
        acc[0].addp(q2 * v[0].y, v[0].y);
    }
    template <typename T> __device__ static void apply(const ModeK<T>& m, int kx, int ky, typename CT<T>::t (&v)[1]) {
        lap_apply(m, kx, ky, v);
    }
    template <typename T> __device__ static void finalize(const Desc<T>& d, const double* tot) {
        Ctrl* c = d.ctrl;
        const double pJp = c->pf_pap + d.k.kappa * tot[0] * d.k.inv_n;
        c->pJp = pJp;
        if (!(pJp > 0.0)) {
            c->pf_break = 1;
            c->pf_alpha = 0.0;
        } else {
            c->pf_alpha = -c->pf_rp / pJp;
        }
    }
};

// sum a p'^2 and r'.p' of the next direction p' = -r' + beta p from S1..S4 (see above)
__device__ __forceinline__ void pf_next_dir(Ctrl* c, const double* S) {
    const double b = c->pf_beta;
    c->pf_pap = S[0] - 2.0 * b * S[1] + b * b * S[2];
    c->pf_rp = -c->pf_rr + b * S[3];
}

// Iteration end shared by the fused iterate kernel (recurrence residual) and the
// explicit residual kernel: beta, ||r||, active count and the stopping decision.
template <typename T>
__device__ __forceinline__ void pf_finish(const Desc<T>& d, Ctrl* c, double rr, double rro, double nact, bool full) {
    if (!d.k.pf_precond) {   // (the preconditioned variant takes beta from the z pass)
        double den = -c->pf_rp;   // = alpha p.Jp
        c->pf_beta = den != 0.0 ? (rr - rro) / den : 0.0;
    }
    c->pf_rr = rr;
    c->pf_it += 1;
    c->n_active = (int)nact;
    double rn = sqrt(rr);
    bool conv = false;
    if (full) {
        c->pf_full_iters += 1;
        c->pf_since_full = 0;
        conv = rn <= c->pf_target;
        // FP32: a confirming evaluation that improved little on the previous explicit
        // residual has reached the rounding level of Jv - b
        if (!conv && sizeof(T) == 4 && c->pf_confirm && rn >= 0.5 * c->pf_last_full) conv = true;
        c->pf_last_full = rn;
        if (rn < c->pf_best) { c->pf_best = rn; c->pf_best_it = c->pf_it; }
    } else {
        c->pf_since_full += 1;
        if (rn <= c->pf_target) c->pf_force = 1;   // confirm with an explicit residual first
    }
    // FP32 safety net: no new smallest explicit residual for PF_STALL iterations
    bool stalled = sizeof(T) == 4 && c->pf_it - c->pf_best_it >= PF_STALL;
    if (conv || stalled || c->pf_it >= d.k.max_pf || c->pf_break) {
        if (!conv && !stalled && !c->pf_break) c->status |= 2;
        c->pf_b = 1;
    } else {
        c->pf_b = 0;
    }
}

// Fused iterate (elementwise): v = max(v + alpha p, v_con) with the bound flag,
// and the residual by recurrence R_new = R + alpha J p, which is exact when the
// projection changed no value.  The active set {bound and R > 0} zeroes r.  When
// some value was clamped (or every PF_REFRESH iterations, or to confirm
// convergence) the finalizer leaves the iteration to the explicit J v - b
// evaluation that follows; otherwise it commits the new residual buffer.
constexpr int PF_REFRESH = 32;

template <typename T>
struct FPfB1 {
    static constexpr int NR = 4;
    struct Ctx { T alpha; double alpha_d; const T* ro; T* rn; };
    __device__ static bool skip(const Desc<T>& d) { return ldflag(&d.ctrl->pf_a); }
    __device__ static Ctx prep(const Desc<T>& d) {
        int sel = ldflag(&d.ctrl->pf_rsel);
        const double a = ldd(&d.ctrl->pf_alpha);
        return Ctx{T(a), a, pf_r(d, sel), pf_r(d, sel ^ 1)};
    }
    struct In { T v, p, vc, R, Jp, ro; };
    __device__ static In load(const Desc<T>& d, const Ctx& c, size_t i) {
        return In{d.th[0][i], d.th[2][i], d.r[2][i], d.lap[i], d.q[0][i], c.ro[i]};
    }
    __device__ static void pixel(const Desc<T>& d, const Ctx& c, size_t i, const In& a, Acc<T>* acc) {
        T x = a.v + c.alpha * a.p;
        if (x < a.vc) { x = a.vc; acc[0].count(T(1)); }
        d.th[0][i] = x;
        const bool at = (x == a.vc);
        T rn = a.R + c.alpha * a.Jp;
        d.lap[i] = rn;
        bool pos = false;
        if (at) {   // the sign only matters at the bound
            if constexpr (sizeof(T) == 8) {
                pos = rn > T(0);
            } else {
                // the FP32 recurrence differs from R + alpha_d J p (exact operands, FP64
                // alpha) by at most 3 units of 2^-24 of |R| + |alpha J p|: beyond 4e-7 of
                // that the FP32 sign is the FP64 sign, below it the sign is taken in FP64
                T mag = fabs(a.R) + fabs(c.alpha * a.Jp);
                if (fabs(rn) > T(4e-7) * mag) pos = rn > T(0);
                else pos = recur_positive_fp64(a.R, c.alpha_d, a.Jp);
            }
        }
        const bool active = at && pos;
        if (active) rn = T(0);
        c.rn[i] = rn;
        d.flags[i] = (uint8_t)((at ? 1 : 0) | (active ? 2 : 0));
        acc[1].addp(rn, rn);
        acc[2].addp(rn, a.ro);
        if (active) acc[3].count(T(1));
    }
    __device__ static void finalize(const Desc<T>& d, const double* tot) {
        Ctrl* c = d.ctrl;
        const bool clamped = tot[0] > 0.0;
        if (clamped) c->pf_clamp_iters += 1;   // iterations in which the clamp changed v
        // a recurrence residual that meets the tolerance is confirmed by the explicit
        // J v - b of this same iteration, so that the solve stops at the iteration at
        // which Algorithm 1's explicit residual first meets it
        const bool rec_conv = sqrt(tot[1]) <= c->pf_target;
        const bool full = clamped || rec_conv || c->pf_force || c->pf_since_full + 1 >= PF_REFRESH;
        c->pf_full = full;
        c->pf_confirm = rec_conv || c->pf_force;
        c->pf_force = 0;
        if (!full) {
            c->pf_rsel ^= 1;
            pf_finish(d, c, tot[1], tot[2], tot[3], false);
        }
    }
};

template <typename T>
struct FPfA3B {   // J p from the column pass's lap p, then the iterate of FPfB1
    static constexpr int NR = 8;
    struct Ctx { T kappa; T alpha; double alpha_d; const T* ro; T* rn; };
    __device__ static bool skip(const Desc<T>& d) { return ldflag(&d.ctrl->pf_a); }
    __device__ static Ctx prep(const Desc<T>& d) {
        const int sel = ldflag(&d.ctrl->pf_rsel);
        const double a = ldd(&d.ctrl->pf_alpha);
        return Ctx{T(d.k.kappa), T(a), a, pf_r(d, sel), pf_r(d, sel ^ 1)};
    }
    struct In { T p, a, v, vc, R, ro; };
    __device__ static In load(const Desc<T>& d, const Ctx& c, size_t i) {
        return In{d.th[2][i], d.r[0][i], d.th[0][i], d.r[2][i], d.lap[i], c.ro[i]};
    }
    __device__ static void pixel(const Desc<T>& d, const Ctx& c, size_t i, const In& a, T (&lp)[1], Acc<T>* acc) {
        const T Jp = a.a * a.p - c.kappa * lp[0];
        T x = a.v + c.alpha * a.p;
        if (x < a.vc) { x = a.vc; acc[0].count(T(1)); }
        d.th[0][i] = x;
        const bool at = (x == a.vc);
        T rn = a.R + c.alpha * Jp;
        d.lap[i] = rn;
        bool pos = false;
        if (at) {   // the sign only matters at the bound (FP64 where FP32 is not decisive, as FPfB1)
            if constexpr (sizeof(T) == 8) {
                pos = rn > T(0);
            } else {
                T mag = fabs(a.R) + fabs(c.alpha * Jp);
                if (fabs(rn) > T(4e-7) * mag) pos = rn > T(0);
                else pos = recur_positive_fp64(a.R, c.alpha_d, Jp);
            }
        }
        const bool active = at && pos;
        if (active) rn = T(0);
        c.rn[i] = rn;
        d.flags[i] = (uint8_t)((at ? 1 : 0) | (active ? 2 : 0));
        acc[1].addp(rn, rn);
        acc[2].addp(rn, a.ro);
        if (active) acc[3].count(T(1));
        if (!active) {   // sums of the next direction (free pixels)
            const T ar = a.a * rn;
            acc[4].addp(ar, rn);
            acc[5].addp(ar, a.p);
            acc[6].addp(a.a * a.p, a.p);
            acc[7].addp(rn, a.p);
        }
    }
    __device__ static void finalize(const Desc<T>& d, const double* tot) {
        FPfB1<T>::finalize(d, tot);
        if (!d.ctrl->pf_full) pf_next_dir(d.ctrl, tot + 4);   // else the explicit residual pass does it
    }
};

template <typename T>
struct FPfVIn {   // input v for the explicit J v (only when pf_full)
    static constexpr int NR = 0;
    using Ctx = NoCtx;
    __device__ static bool skip(const Desc<T>& d) { return ldflag(&d.ctrl->pf_a) || !ldflag(&d.ctrl->pf_full); }
    __device__ static Ctx prep(const Desc<T>&) { return Ctx{}; }
    __device__ static void pixel(const Desc<T>& d, const Ctx&, size_t i, T (&v)[1], Acc<T>*) { v[0] = d.th[0][i]; }
    __device__ static void finalize(const Desc<T>&, const double*) {}
};

struct FColLapPFFull {
    template <typename T> __device__ static bool skip(const Desc<T>& d) {
        return ldflag(&d.ctrl->pf_a) || !ldflag(&d.ctrl->pf_full);
    }
    template <typename T> __device__ static void apply(const ModeK<T>& m, int kx, int ky, typename CT<T>::t (&v)[1]) {
        lap_apply(m, kx, ky, v);
    }
};

template <typename T>
struct FPfB3 {   // explicit R = J v - b, active set {bound and R > 0}, beta, convergence (only when pf_full)
    static constexpr int NR = 7;
    struct Ctx { T kappa; double kd; const T* ro; T* rn; };
    __device__ static bool skip(const Desc<T>& d) { return ldflag(&d.ctrl->pf_a) || !ldflag(&d.ctrl->pf_full); }
    __device__ static Ctx prep(const Desc<T>& d) {
        const int sel = ldflag(&d.ctrl->pf_rsel);
        return Ctx{T(d.k.kappa), d.k.kappa, pf_r(d, sel), pf_r(d, sel ^ 1)};
    }
    struct In { T ro, x, a, b, p; uint8_t fl; };
    __device__ static In load(const Desc<T>& d, const Ctx& c, size_t i) {
        return In{c.ro[i], d.th[0][i], d.r[0][i], d.r[1][i], d.th[2][i], d.flags[i]};
    }
    __device__ static void pixel(const Desc<T>& d, const Ctx& c, size_t i, const In& in, T (&v)[1], Acc<T>* acc) {
        const T ro = in.ro, x = in.x, a = in.a, b = in.b, kl = c.kappa * v[0];
        T rn = a * x - kl - b;
        d.lap[i] = rn;
        const bool at = in.fl & 1;
        bool pos = false;
        if (at) {   // the sign only matters at the bound
            if constexpr (sizeof(T) == 8) {
                pos = rn > T(0);
            } else {
                // FP32 residual; decide its sign in FP64 from the same FP32 operands when it
                // is within rounding of zero (otherwise the FP32 sign is already exact)
                T mag = fabs(a * x) + fabs(kl) + fabs(b);
                if (fabs(rn) > T(4e-7) * mag) pos = rn > T(0);
                else pos = resid_positive_fp64(a, x, c.kd, v[0], b);
            }
        }
        const bool active = at && pos;
        if (active) rn = T(0);
        c.rn[i] = rn;   // beside the previous residual (kept for the preconditioned beta)
        d.flags[i] = (uint8_t)((at ? 1 : 0) | (active ? 2 : 0));
        acc[0].addp(rn, rn);
        acc[1].addp(rn, ro);
        if (active) acc[2].count(T(1));
        if (!active) {   // sums of the next direction (free pixels; used by the three-pass iteration)
            const T ar = a * rn;
            acc[3].addp(ar, rn);
            acc[4].addp(ar, in.p);
            acc[5].addp(a * in.p, in.p);
            acc[6].addp(rn, in.p);
        }
    }
    __device__ static void finalize(const Desc<T>& d, const double* tot) {
        d.ctrl->pf_rsel ^= 1;
        pf_finish(d, d.ctrl, tot[0], tot[1], tot[2], true);
        pf_next_dir(d.ctrl, tot + 3);
    }
};

// Algorithm 4 lines 12-14: phi_{n+1} = phi_n + v, sigma-bar(eps_n, phi_{n+1}), C-bar,
// ||dphi||_1, F_e, strain increment.
template <typename T>
struct FPost {
    static constexpr int NR = 5;
    struct Ctx { T eb[3]; LameC<T> lm; };
    __device__ static bool skip(const Desc<T>&) { return false; }
    __device__ static Ctx prep(const Desc<T>& d) {
        Ctx c{{}, LameC<T>(d)};
        for (int k = 0; k < 3; ++k) c.eb[k] = T(ldd(&d.ctrl->eps_bar[k]));
        return c;
    }
    __device__ static void pixel(const Desc<T>& d, const Ctx& c, size_t i, Acc<T>* acc) {
        T v = d.th[0][i];
        T ph = d.phi[i] + v;
        d.phi[i] = ph;
        T lam, mu;
        c.lm.at(d, i, lam, mu);
        T xx = c.eb[0] + d.eps[0][i], yy = c.eb[1] + d.eps[1][i], xy = c.eb[2] + d.eps[2][i];
        T h = hdeg(ph);
        T s[3];
        stress(d.k.split, xx, yy, xy, h, lam, mu, s);
        acc[0].add(s[0]);
        acc[1].add(s[1]);
        acc[2].add(s[2]);
        acc[3].add(energy(d.k.split, xx, yy, xy, h, lam, mu));
        acc[4].add(fabs(v));
    }
    __device__ static void finalize(const Desc<T>& d, const double* tot) {
        Ctrl* c = d.ctrl;
        const Consts& k = d.k;
        double sb[3] = {tot[0] * k.inv_n, tot[1] * k.inv_n, tot[2] * k.inv_n};
        double eb[3] = {c->eps_bar[0], c->eps_bar[1], c->eps_bar[2]};
        // C-bar at the largest |eps_bar| component, row-major order xx, xy, yy
        int j = 0;
        double m = fabs(eb[0]);
        if (fabs(eb[2]) > m) { j = 2; m = fabs(eb[2]); }
        if (fabs(eb[1]) > m) { j = 1; m = fabs(eb[1]); }
        double Cb = eb[j] != 0.0 ? sb[j] / eb[j] : INFINITY;
        double dphi = k.L1_scale * tot[4];
        for (int q = 0; q < 3; ++q) { c->sig_bar[q] = sb[q]; c->rep_eps_bar[q] = eb[q]; }
        c->C_bar = Cb;
        c->dphi = dphi;
        c->Fe = tot[3] * k.dA;
        c->incremented = c->post_mode == 0 && dphi < k.dphi_min;
        if (c->incremented)
            for (int q = 0; q < 3; ++q) c->eps_bar[q] = eb[q] + k.d_eps_bar[q];
        c->broken = Cb < k.C_broken;
    }
};

// aux = phi_con(phi) (the constraint of an alternating-minimisation increment),
// aux = phi (time-step retry point), phi = aux (retry)
template <typename T, int MODE>
struct FAux {
    static constexpr int NR = 0;
    using Ctx = NoCtx;
    __device__ static bool skip(const Desc<T>&) { return false; }
    __device__ static Ctx prep(const Desc<T>&) { return Ctx{}; }
    __device__ static void pixel(const Desc<T>& d, const Ctx&, size_t i, Acc<T>*) {
        if (MODE == 0) {
            T ph = d.phi[i];
            d.aux[i] = (d.k.irrev == CRACK_SET) ? (ph >= T(d.k.crack_thr) ? ph : T(0)) : ph;
        } else if (MODE == 1) {
            d.aux[i] = d.phi[i];
        } else {
            d.phi[i] = d.aux[i];
        }
    }
    __device__ static void finalize(const Desc<T>&, const double*) {}
};

}  // namespace pff
