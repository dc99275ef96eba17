// k_cluster.cu -- the mechanics sub-problem (Sec. 3.1.1: Newton over CG on the
// Fourier-Galerkin equations P sigma = 0) of FP32 512 x 512 problems, one
// thread-block cluster of 16 CTAs per problem, the whole Newton-CG solve in one
// launch.
//
// Data placement.  The half spectrum of the three tensor components (kx < 256;
// the Nyquist column kx = 256 and row ky = 256 are zeroed by the projection)
// is held in the cluster's shared memory, 192 KB per CTA, and never goes to
// HBM.  CTA c owns the real-space rows y in [32c, 32c + 32) and the spectral
// columns kx in [16c, 16c + 16).  Its buffer X_c is split into 16 slots of
// 3 x 32 x 16 complex values; slot s of X_c holds the modes (kx in c's columns,
// ky in [32s, 32s + 32)).  The forward row FFTs of CTA c write their modes of
// column block s straight into slot c of CTA s (distributed shared memory), and
// the inverse row FFTs read them back from the same place: during a row phase
// only CTA c touches slot c of any CTA, so the row phases need no cluster
// barrier of their own.
//
// One CG iteration = one row phase + one column phase:
//   row phase (each CTA, 2 rows at a time): read q = A p of the previous
//     iteration (inverse row FFT of the Gamma-projected modes), update
//     theta += alpha p, r -= alpha q, p = r + beta p (stored to HBM), the
//     tangent tau = C_m : p, forward row FFT of tau into the column owners;
//     partial r.r, p.tau, r.tau.
//   cluster barrier
//   column phase (each CTA, its 16 columns): FFT along y, Gamma(q) scaled by
//     1/(nx ny), partial |Gamma tau|^2 (Parseval: q.q), inverse FFT along y.
//   cluster barrier
// Every CG iterate stays in range(P) (P = F^-1 Gamma F, an orthogonal
// projection), so p.Ap = p.P tau = p.tau and r.Ap = r.tau; with q.q from the
// modes, alpha = r.r / p.Ap and beta = (r.r - 2 alpha r.Ap + alpha^2 q.q) / r.r
// are known before the next row phase, which therefore applies the update, the
// new tangent and the next forward FFT in one pass over the pixels.  The
// stopping test uses the explicit r.r of the updated residual (as the
// per-kernel path does).
//
// Reductions: per thread compensated FP32 pairs, per CTA double-float, the CTA
// totals as doubles in each CTA's shared memory (double-buffered by iteration
// parity); after the barrier every CTA sums the 16 totals in rank order in
// FP64, so all CTAs take identical decisions and leave their loops together.
// The only waits are the hardware cluster barriers, which every thread of
// every CTA reaches the same number of times.
#include <cooperative_groups.h>

#include "kernels.cuh"
#include "launch.h"

namespace cgr = cooperative_groups;

namespace pff {
namespace {

constexpr int QN = 512;                   // grid size (nx = ny)
constexpr int QM = QN / 2;                // row FFT length (complex)
constexpr int QCS = 16;                   // CTAs per cluster
constexpr int QRPC = QN / QCS;            // rows per CTA, ky per slot (32)
constexpr int QKPC = QM / QCS;            // spectral columns per CTA (16)
constexpr int QNT = 256;                  // threads per CTA
constexpr int QRS = 2;                    // rows per row step
constexpr int QNSEQ = 3 * QRS;            // row FFT sequences per step
constexpr int QSP = padded_len(QM) + 2;   // staging pitch (complex values)
constexpr int QX = QCS * 3 * QRPC * QKPC; // spectrum values per CTA (24576)
constexpr int QCW = QNT / 64;              // columns per column round (64 threads per column)
constexpr size_t QSMEM = (size_t)(QX + QNSEQ * QSP + padded_len(QN)) * sizeof(float2);
constexpr int QPPT = QRS * QN / QNT;      // pixels per thread per row step
static_assert(QPPT * QNT == QRS * QN && QN % QNT == 0, "whole rows per thread pass");
static_assert(QKPC % QCW == 0, "whole column rounds");

// Position of (slot, component, t, column i) in X.  The column index is swizzled
// (i ^ 4 ((t + t/8) mod 4)) so that the accesses of the column FFT -- a warp
// holds 4 or 8 columns and 8 or 4 values of t that are consecutive or 8 apart --
// spread over all shared-memory banks; a row segment (the 16 values of one t)
// stays within one 128-byte line.
__device__ __forceinline__ int xpos(int slot, int comp, int t, int i) {
    return ((slot * 3 + comp) * QRPC + t) * QKPC + (i ^ (((t + (t >> 3)) & 3) << 2));
}
// element ky of the column (comp, i) of this CTA
__device__ __forceinline__ int cpos(int comp, int i, int ky) { return xpos(ky >> 5, comp, ky & 31, i); }

enum { MODE_RESID = 0, MODE_INIT = 1, MODE_CG = 2 };

struct Dec {            // decisions shared by the threads of a CTA
    float alpha, beta;
    int stop;
};

// Warp shuffles then warp 0: the CTA total of NR double-float values as doubles
// (valid in thread 0).
template <int NR>
__device__ __forceinline__ void cta_reduce(const Acc<float>* acc, double (&out)[NR], DF (*wbuf)[QNT / 32]) {
    using O = RedOps<DF>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        DF x = acc[k].df();
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x = O::add(x, O::shfl(x, o));
        if (lane == 0) wbuf[k][warp] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NR; ++k) {
            DF x = wbuf[k][0];
            for (int w = 1; w < QNT / 32; ++w) x = O::add(x, wbuf[k][w]);
            out[k] = O::total(x);
        }
    }
}

// cluster-wide FP64 sums of the CTA totals part[par][k0 .. k0+n) in rank order (thread 0)
__device__ __forceinline__ void cluster_sums(cgr::cluster_group& cl, double (*part)[4], int par, int k0, int n,
                                             double* out) {
    for (int k = 0; k < n; ++k) out[k] = 0.0;
    for (int r = 0; r < QCS; ++r) {
        const double* rp = cl.map_shared_rank(&part[par][0], r);
        for (int k = 0; k < n; ++k) out[k] += rp[k0 + k];
    }
}

// ---------------------------------------------------------------- column phase
template <bool INV>
__device__ __forceinline__ void fft512_x(float2 (&u)[3][8], int n0, int t, float2* X, int i, const float2* tws) {
    float2 w[8];
    tw8<float2, INV>(tws, n0, w);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        dft8<float2, INV>(u[c]);
#pragma unroll
        for (int r = 1; r < 8; ++r) u[c][r] = cmul(u[c][r], w[r]);
    }
    __syncthreads();   // earlier readers of these positions are done
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int k1 = 0; k1 < 8; ++k1) X[cpos(c, i, 64 * k1 + n0)] = u[c][k1];
    __syncthreads();
    const int k1 = t >> 3, a = t & 7;
    tw8<float2, INV>(tws, 8 * a, w);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
#pragma unroll
        for (int b = 0; b < 8; ++b) u[c][b] = X[cpos(c, i, 64 * k1 + a + 8 * b)];
        dft8<float2, INV>(u[c]);
#pragma unroll
        for (int r = 1; r < 8; ++r) u[c][r] = cmul(u[c][r], w[r]);
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int cc = 0; cc < 8; ++cc) X[cpos(c, i, 64 * k1 + a + 8 * cc)] = u[c][cc];
    __syncthreads();
#pragma unroll
    for (int c = 0; c < 3; ++c) {
#pragma unroll
        for (int aa = 0; aa < 8; ++aa) u[c][aa] = X[cpos(c, i, 64 * k1 + aa + 8 * a)];
        dft8<float2, INV>(u[c]);
    }
}

// FFT along y of this CTA's 16 columns (two rounds of 8), the projection Gamma
// scaled by 1/(nx ny), the inverse FFT; acc += sum over the modes of
// w(kx) |Gamma tau|_F^2 (w = 1 at kx = 0, else 2: the half spectrum).
__device__ __noinline__ void column_phase(float2* X, const float2* twc, const ModeK<float>& mk, int rank,
                                             Acc<float>& acc) {
    const int j = threadIdx.x % QCW, t = threadIdx.x / QCW;
    for (int round = 0; round < QKPC / QCW; ++round) {
        const int i = round * QCW + j;
        const int kx = rank * QKPC + i;
        float2 u[3][8];
        __syncthreads();   // the previous round's last stores are done
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int m = 0; m < 8; ++m) u[c][m] = X[cpos(c, i, t + 64 * m)];
        fft512_x<false>(u, t, t, X, i, twc);
        const int k1 = t >> 3, cc = t & 7;
        const float wk = kx == 0 ? 1.f : 2.f;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            float2 v[3] = {u[0][e], u[1][e], u[2][e]};
            gamma_apply(mk, kx, k1 + 8 * cc + 64 * e, v);
            acc.addp(wk * v[0].x, v[0].x); acc.addp(wk * v[0].y, v[0].y);
            acc.addp(wk * v[1].x, v[1].x); acc.addp(wk * v[1].y, v[1].y);
            acc.addp(2.f * wk * v[2].x, v[2].x); acc.addp(2.f * wk * v[2].y, v[2].y);
            u[0][e] = v[0]; u[1][e] = v[1]; u[2][e] = v[2];
        }
        const int tp = k1 + 8 * cc;
        fft512_x<true>(u, tp, t, X, i, twc);
        __syncthreads();   // all reads of the last stage are done
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int e = 0; e < 8; ++e) X[cpos(c, i, tp + 64 * e)] = u[c][e];
    }
}

// ---------------------------------------------------------------- row phase
struct RowCtx {
    float alpha, beta;
    float eb[3];
    LameC<float> lm;
    int split;
    int fold;           // RESID: eps* += theta first (Newton rounds after the first)
};

struct PixIn { float th[3], r[3], p[3], e[3], phi, E; };

// One row phase: the CTA's 32 rows in steps of QRS.  acc: r.r, p.tau, r.tau.
template <int MODE>
__device__ __noinline__ void row_phase(cgr::cluster_group& cl, const Desc<float>& d, const RowCtx& cx,
                                          float2* X, float2* buf, int rank, Acc<float>* acc) {
    float* rb = reinterpret_cast<float*>(buf);
    const float2* twr = d.tw + QM;    // FFT table of length QM (global, L1-cached)
    const float2* twN = d.tw + QN;    // exp(-2 pi i k / QN), k <= QM
    for (int t0 = 0; t0 < QRPC; t0 += QRS) {
        const int y0 = rank * QRPC + t0;
        // epilogue loads first: they are in flight during the gather and the FFT
        // (pixel j of this thread: row j*QNT/QN, column x = (j*QNT) % QN + thread)
        PixIn in[QPPT];
#pragma unroll
        for (int r = 0; r < QPPT; ++r) {
            const int pl = r * QNT + threadIdx.x;
            const size_t px = (size_t)(y0 + pl / QN) * QN + pl % QN;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                in[r].e[k] = d.eps[k][px];
                if constexpr (MODE == MODE_CG) {
                    in[r].th[k] = d.th[k][px];
                    in[r].r[k] = d.r[k][px];
                    in[r].p[k] = d.p[k][px];
                }
                if constexpr (MODE == MODE_RESID) {
                    if (cx.fold) in[r].th[k] = d.th[k][px];
                }
            }
            in[r].phi = d.phi[px];
            in[r].E = d.E[px];
        }
        __syncthreads();   // the staging buffer is free (previous step done)
        if constexpr (MODE != MODE_RESID) {
            // gather the rows' modes kx < QM from their column owners (kx = QM is zero)
            for (int idx = threadIdx.x; idx < QNSEQ * QM; idx += QNT) {
                const int s = idx / QM, k = idx % QM;
                const int comp = s / QRS, r = s % QRS;
                const float2* src = cl.map_shared_rank(X, k / QKPC);
                buf[s * QSP + pidx(k)] = src[xpos(rank, comp, t0 + r, k % QKPC)];
            }
            for (int s = threadIdx.x; s < QNSEQ; s += QNT) buf[s * QSP + pidx(QM)] = make_float2(0.f, 0.f);
            __syncthreads();
            // complex-to-real pre-processing: Z[k] = A + i B with A = X[k] + conj(X[M-k]),
            // B = (X[k] - conj(X[M-k])) e^{+2 pi i k/N}
            float2 z[QNSEQ * QM / QNT];
#pragma unroll
            for (int u = 0; u < QNSEQ * QM / QNT; ++u) {
                const int tt = threadIdx.x + u * QNT;
                const int s = tt / QM, k = tt % QM;
                float2 xk = buf[s * QSP + pidx(k)], xm = buf[s * QSP + pidx(QM - k)];
                if (k == 0) { xk.y = 0.f; xm.y = 0.f; }
                xm.y = -xm.y;
                const float2 A = cadd(xk, xm);
                const float2 B = cmulc(csub(xk, xm), __ldg(&twN[k]));
                z[u] = make_float2(A.x - B.y, A.y + B.x);
            }
            __syncthreads();
#pragma unroll
            for (int u = 0; u < QNSEQ * QM / QNT; ++u) {
                const int tt = threadIdx.x + u * QNT;
                buf[(tt / QM) * QSP + pidx(tt % QM)] = z[u];
            }
            __syncthreads();
            fft_smem<float, QM, QNSEQ, QSP, QNT, true, false>(buf, twr);
        }
        // per pixel
#pragma unroll
        for (int j = 0; j < QPPT; ++j) {
            const int pl = j * QNT + threadIdx.x;
            const int r = pl / QN, x = pl % QN;
            const size_t px = (size_t)(y0 + r) * QN + x;
            const PixIn& a = in[j];
            float lam = cx.lm.lc * a.E, mu = cx.lm.mc * a.E;
            const float h = hdeg(a.phi);
            float out[3];
            if constexpr (MODE == MODE_RESID) {
                float e[3] = {a.e[0], a.e[1], a.e[2]};
                if (cx.fold) {
#pragma unroll
                    for (int k = 0; k < 3; ++k) { e[k] += a.th[k]; d.eps[k][px] = e[k]; }
                }
                stress(cx.split, cx.eb[0] + e[0], cx.eb[1] + e[1], cx.eb[2] + e[2], h, lam, mu, out);
            } else {
                float q[3], rr[3], p[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) q[k] = rb[(k * QRS + r) * 2 * QSP + ridx(x)];
                if constexpr (MODE == MODE_INIT) {   // r = p = -R, theta = 0 (CG start of a Newton round)
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        rr[k] = -q[k];
                        p[k] = -q[k];
                        d.r[k][px] = rr[k];
                        d.p[k][px] = p[k];
                        d.th[k][px] = 0.f;
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        d.th[k][px] = a.th[k] + cx.alpha * a.p[k];
                        rr[k] = a.r[k] - cx.alpha * q[k];
                        p[k] = rr[k] + cx.beta * a.p[k];
                        d.r[k][px] = rr[k];
                        d.p[k][px] = p[k];
                    }
                }
                tangent(cx.split, cx.eb[0] + a.e[0], cx.eb[1] + a.e[1], cx.eb[2] + a.e[2], h, lam, mu,
                        p[0], p[1], p[2], out);
                wdot(acc[0], rr[0], rr[1], rr[2], rr[0], rr[1], rr[2]);
                wdot(acc[1], p[0], p[1], p[2], out[0], out[1], out[2]);
                wdot(acc[2], rr[0], rr[1], rr[2], out[0], out[1], out[2]);
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) rb[(k * QRS + r) * 2 * QSP + ridx(x)] = out[k];
        }
        __syncthreads();
        fft_smem<float, QM, QNSEQ, QSP, QNT, false, false>(buf, twr);
        // real-to-complex post-processing X[k] = Xe[k] + W_N^k Xo[k] (k < QM; the Nyquist
        // mode kx = QM is dropped: the projection zeroes it), written to the column owner
        for (int idx = threadIdx.x; idx < QNSEQ * QM; idx += QNT) {
            const int s = idx / QM, k = idx % QM;
            const int comp = s / QRS, r = s % QRS;
            float2 zk = buf[s * QSP + pidx(k)];
            float2 zm = buf[s * QSP + pidx(k == 0 ? 0 : QM - k)];
            zm.y = -zm.y;
            const float2 e = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y + zm.y));
            const float2 o = make_float2(0.5f * (zk.y - zm.y), -0.5f * (zk.x - zm.x));
            float2* dst = cl.map_shared_rank(X, k / QKPC);
            dst[xpos(rank, comp, t0 + r, k % QKPC)] = cadd(e, cmul(__ldg(&twN[k]), o));
        }
    }
}

// eps* += theta on this CTA's rows (the single Newton step of a linear model)
__device__ __forceinline__ void fold_rows(const Desc<float>& d, int rank) {
    for (int idx = threadIdx.x; idx < QRPC * QN; idx += QNT) {
        const size_t px = (size_t)rank * QRPC * QN + idx;
#pragma unroll
        for (int k = 0; k < 3; ++k) d.eps[k][px] += d.th[k][px];
    }
}

__global__ void __launch_bounds__(QNT, 1) k_mech_cluster(const Desc<float>* __restrict__ descs) {
    cgr::cluster_group cl = cgr::this_cluster();
    const int rank = (int)cl.block_rank();
    const Desc<float>& d = descs[blockIdx.x / QCS];
    Ctrl* ctrl = d.ctrl;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* X = reinterpret_cast<float2*>(smem_raw);
    float2* buf = X + QX;
    float2* twc = buf + QNSEQ * QSP;
    __shared__ double s_part[2][4];           // this CTA's totals, by iteration parity
    __shared__ DF s_w[3][QNT / 32];
    __shared__ Dec s_dec;
    __shared__ RowCtx s_cx;

    for (int k = threadIdx.x; k < QN; k += QNT) twc[pidx(k)] = d.tw[QN + k];
    const ModeK<float> mk(d);
    const Consts& K = d.k;
    const bool linear = contact_of(K.split) == ISOTROPIC;
    if (threadIdx.x == 0) {
        RowCtx c;
        c.alpha = 0.f; c.beta = 0.f;
        for (int k = 0; k < 3; ++k) c.eb[k] = (float)ldd(&ctrl->eps_bar[k]);
        c.lm = LameC<float>(d);
        c.split = K.split;
        c.fold = 0;
        s_cx = c;
    }
    // every CTA of the cluster is running before any distributed shared memory access
    cl.sync();

    // target ||C0(E):eps_bar|| tol (as the per-kernel path)
    const double eb0 = ldd(&ctrl->eps_bar[0]), eb1 = ldd(&ctrl->eps_bar[1]), eb2 = ldd(&ctrl->eps_bar[2]);
    const double trb = eb0 + eb1;
    const double s0 = K.lam_c * trb + 2.0 * K.mu_c * eb0, s1 = K.lam_c * trb + 2.0 * K.mu_c * eb1,
                 s2 = 2.0 * K.mu_c * eb2;
    const double target = K.mech_tol * sqrt(ldd(&ctrl->sumE2)) * sqrt(s0 * s0 + s1 * s1 + 2.0 * s2 * s2);
    const double nn = (double)QN * (double)QN;

    int par = 0;
    int newton_it = 0, cg_total = 0, cg_it = 0, status = 0, cg_break = 0;
    double R2 = 0.0, rr = 0.0, cg_target = 0.0;
    for (;;) {
        // ---- Newton residual R = P sigma(eps_bar + eps*) and ||R||
        row_phase<MODE_RESID>(cl, d, s_cx, X, buf, rank, nullptr);
        cl.sync();
        {
            Acc<float> acc;
            column_phase(X, twc, mk, rank, acc);
            double tot[1];
            cta_reduce<1>(&acc, tot, s_w);
            if (threadIdx.x == 0) s_part[par][3] = tot[0];
        }
        cl.sync();
        if (threadIdx.x == 0) {
            double v[1];
            cluster_sums(cl, s_part, par, 3, 1, v);
            R2 = v[0] * nn;
            const double rn = sqrt(R2);
            int stop = 0;
            if (rn <= target || newton_it >= K.max_newton) {
                if (rn > target) status |= 1;
                stop = 1;
            } else {
                cg_target = linear ? target : fmax(target, K.mech_cg_rtol * rn);
                newton_it += 1;
            }
            s_dec.stop = stop;
        }
        __syncthreads();
        par ^= 1;
        if (s_dec.stop) break;
        // ---- CG on P C_m theta = -R from theta = 0
        cg_it = 0;
        cg_break = 0;
        Acc<float> acc[3];
        row_phase<MODE_INIT>(cl, d, s_cx, X, buf, rank, acc);
        for (;;) {
            double tot[3];
            cta_reduce<3>(acc, tot, s_w);
            if (threadIdx.x == 0) { s_part[par][0] = tot[0]; s_part[par][1] = tot[1]; s_part[par][2] = tot[2]; }
            cl.sync();
            // stopping test on the explicit r.r of the updated residual
            if (threadIdx.x == 0) {
                double v[1];
                cluster_sums(cl, s_part, par, 0, 1, v);
                rr = v[0];
                s_dec.stop = (sqrt(rr) <= cg_target || cg_it >= K.max_cg || cg_break) ? 1 : 0;
                if (s_dec.stop && !(sqrt(rr) <= cg_target) && !cg_break) status |= 1;
            }
            __syncthreads();
            if (s_dec.stop) break;
            Acc<float> accq;
            column_phase(X, twc, mk, rank, accq);
            {
                double tq[1];
                cta_reduce<1>(&accq, tq, s_w);
                if (threadIdx.x == 0) s_part[par][3] = tq[0];
            }
            cl.sync();
            if (threadIdx.x == 0) {
                double v[4];
                cluster_sums(cl, s_part, par, 0, 4, v);
                const double pAp = v[1], rAp = v[2], qq = v[3] * nn;
                cg_it += 1;
                cg_total += 1;
                double a = 0.0, b = 0.0;
                if (!(pAp > 0.0)) {
                    cg_break = 1;
                } else {
                    a = rr / pAp;
                    double rn2 = rr - 2.0 * a * rAp + a * a * qq;
                    if (rn2 < 0.0) rn2 = 0.0;
                    b = rr > 0.0 ? rn2 / rr : 0.0;
                }
                s_cx.alpha = (float)a;
                s_cx.beta = (float)b;
            }
            __syncthreads();
            par ^= 1;
#pragma unroll
            for (int k = 0; k < 3; ++k) acc[k] = Acc<float>();
            row_phase<MODE_CG>(cl, d, s_cx, X, buf, rank, acc);
        }
        par ^= 1;
        if (linear) {   // a linear model takes one Newton step (Sec. 3.1.1)
            fold_rows(d, rank);
            break;
        }
        if (threadIdx.x == 0) s_cx.fold = 1;
        __syncthreads();
    }
    if (rank == 0 && threadIdx.x == 0) {
        ctrl->mech_target = target;
        ctrl->R2 = R2;
        ctrl->rr = rr;
        ctrl->cg_target = cg_target;
        ctrl->newton_it = newton_it;
        ctrl->cg_it = cg_it;
        ctrl->cg_total = cg_total;
        ctrl->cg_break = cg_break;
        ctrl->status |= status;
        ctrl->nd_a = 1; ctrl->nd_b = 1;
        ctrl->cg_a = 1; ctrl->cg_b = 1;
        ctrl->needs_fold = 0;
    }
    // no CTA leaves while another may still address its shared memory
    cl.sync();
}

}  // namespace

// Whether the device can run the cluster solve (16 CTAs of QSMEM bytes each,
// one cluster resident at least); evaluated once per process.
bool mech_cluster_supported() {
    static int ok = -1;
    if (ok < 0) {
        ok = 0;
        int dev = 0, cc = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&cc, cudaDevAttrComputeCapabilityMajor, dev);
        if (cc >= 9 &&
            cudaFuncSetAttribute(k_mech_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)QSMEM) == cudaSuccess &&
            cudaFuncSetAttribute(k_mech_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(QCS);
            cfg.blockDim = dim3(QNT);
            cfg.dynamicSmemBytes = QSMEM;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = QCS;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            int n = 0;
            if (cudaOccupancyMaxActiveClusters(&n, (const void*)k_mech_cluster, &cfg) == cudaSuccess && n >= 1) ok = 1;
        }
        cudaGetLastError();
    }
    return ok == 1;
}

// The whole mechanics solve of np FP32 512 x 512 problems (one cluster each) after
// the step's control-block reset.
cudaError_t launch_mech_cluster(const Desc<float>* d, int np, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(QCS * np);
    cfg.blockDim = dim3(QNT);
    cfg.dynamicSmemBytes = QSMEM;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = QCS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_mech_cluster, d);
    count_launch();
    return e;
}

}  // namespace pff
