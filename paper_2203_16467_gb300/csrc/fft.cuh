// fft.cuh -- shared-memory batched FFTs and the three kernel shapes of a
// 2-D spectral operator F^-1 M F (Sec. 3.1: the DFT pair; the normalisation
// 1/(nx ny) is folded into the mode multiplier M):
//   k_row_fwd : per-pixel prologue -> real FFT along x  -> half spectrum S
//   k_col     : FFT along y -> mode multiplier (Gamma or -|2 pi q|^2) -> inverse FFT along y
//   k_row_inv : half spectrum -> real inverse FFT along x -> per-pixel epilogue (+ reductions)
// FFTs are radix-4 Stockham passes (one radix-2 pass first when log2 of the
// length is odd), register staged and in place in shared memory, with
// twiddles from FP64-accurate tables.
#pragma once
#include "common.cuh"

namespace pff {

// Twiddle tables (per device, built on the host in FP64): the table of
// length M sits at offset M and holds exp(-2 pi i j / M), j < M.
constexpr int TW_MAX = 4096;                 // longest transform

constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }
constexpr int pow2floor(int n) { return n <= 1 ? 1 : 2 * pow2floor(n / 2); }
constexpr int cmin(int a, int b) { return a < b ? a : b; }
constexpr int cmax(int a, int b) { return a > b ? a : b; }

template <typename C, bool INV>
__device__ __forceinline__ void dft4(C& a0, C& a1, C& a2, C& a3) {
    C s02 = cadd(a0, a2), d02 = csub(a0, a2), s13 = cadd(a1, a3), d13 = csub(a1, a3);
    // forward: multiply d13 by -i; inverse: by +i
    C t = INV ? C{-d13.y, d13.x} : C{d13.y, -d13.x};
    a0 = cadd(s02, s13);
    a2 = csub(s02, s13);
    a1 = cadd(d02, t);
    a3 = csub(d02, t);
}

// One Stockham pass of radix R over sequences [s0, s0+G) of length M stored at
// buf[s*SP + j]; p = product of the radices of the previous passes.
//   butterfly i in [0, M/R): k = i mod p; inputs x[i + r M/R]; twiddle
//   w^(r k) with w = exp(-+2 pi i/(p R)); outputs y[(i - k) R + k + r p].
template <typename T, int M, int R, int G, int NSEQ, int SP, int NT, bool INV>
__device__ __forceinline__ void stockham_pass(typename CT<T>::t* buf, int s0, int p, const typename CT<T>::t* tw) {
    using C = typename CT<T>::t;
    constexpr int NBS = M / R;           // butterflies per sequence
    constexpr int NB = G * NBS;          // butterflies in the round
    constexpr int PER = (NB + NT - 1) / NT;
    C u[PER][R];
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        int b = threadIdx.x + j * NT;
        int s = s0 + b / NBS, i = b % NBS;
        if ((NB % NT == 0 || b < NB) && s < NSEQ) {
#pragma unroll
            for (int r = 0; r < R; ++r) u[j][r] = buf[s * SP + i + r * NBS];
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        int b = threadIdx.x + j * NT;
        int s = s0 + b / NBS, i = b % NBS;
        if ((NB % NT == 0 || b < NB) && s < NSEQ) {
            int k = i & (p - 1);
            int step = M / (p * R);
#pragma unroll
            for (int r = 1; r < R; ++r) {
                C w = tw[r * k * step];
                u[j][r] = INV ? cmulc(u[j][r], w) : cmul(u[j][r], w);
            }
            if (R == 4) {
                dft4<C, INV>(u[j][0], u[j][1], u[j][2], u[j][3]);
            } else {
                C a = u[j][0], c = u[j][1];
                u[j][0] = cadd(a, c);
                u[j][1] = csub(a, c);
            }
            int o = (i - k) * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) buf[s * SP + o + r * p] = u[j][r];
        }
    }
    __syncthreads();
}

// NSEQ in-place complex FFTs of length M (unnormalised; forward e^-, inverse e^+).
// Sequences are processed in rounds of G; each thread holds up to PERMAX
// radix-4 butterflies of a round in registers (fewer rounds = fewer barriers).
template <typename T, int M, int NSEQ, int SP, int NT, bool INV>
__device__ __forceinline__ void fft_smem(typename CT<T>::t* buf, const typename CT<T>::t* twbase) {
    constexpr int LOG = ilog2(M);
    constexpr int PERMAX = sizeof(T) == 4 ? 6 : 3;
    constexpr int G = cmax(1, cmin(NSEQ, (4 * NT * PERMAX) / M));   // sequences per round
    const typename CT<T>::t* tw = twbase + M;
    for (int s0 = 0; s0 < NSEQ; s0 += G) {
        int p = 1;
        if (LOG & 1) {
            stockham_pass<T, M, 2, G, NSEQ, SP, NT, INV>(buf, s0, 1, tw);
            p = 2;
        }
        for (; p < M; p *= 4) stockham_pass<T, M, 4, G, NSEQ, SP, NT, INV>(buf, s0, p, tw);
    }
}

// ---------------------------------------------------------------------------
// launch geometry
template <typename T, int NX, int NC>
struct RowCfg {
    static constexpr int M = NX / 2;
    // rows per block: about 512 complex values per block so that a 512^2 grid
    // already gives 128+ blocks per component plane
    static constexpr int ROWS = pow2floor(cmax(1, cmin(16, 512 / (NC * M))));   // divides every ny >= 16
    static constexpr int NT = (NC * ROWS * M >= 1024) ? 256 : 128;
    static constexpr int SP = M + 1;                        // pitch (complex), odd to spread banks
    static constexpr int NSEQ = NC * ROWS;
    static constexpr size_t SMEM = (size_t)NSEQ * SP * sizeof(typename CT<T>::t);
};

template <typename T, int NY, int NC>
struct ColCfg {
    static constexpr int CSZ = (int)sizeof(typename CT<T>::t);
    static constexpr int CWMIN = 32 / CSZ;                   // one 32-byte sector per row segment
    // one 32-byte sector per row segment: enough columns per block for full
    // sectors, and as many blocks as possible
    static constexpr int CWE = CWMIN;
    static constexpr int SP = NY + 1;
    static constexpr int NSEQ = NC * CWE;
    static constexpr int NT = (NSEQ * NY >= 8192) ? 512 : (NSEQ * NY >= 2048 ? 256 : 128);
    static constexpr size_t SMEM = (size_t)NSEQ * SP * CSZ;
};

constexpr int WP_ALIGN = 16;   // spectral row pitch multiple (largest column tile)

// Staging of M+1 spectrum values per sequence in a buffer of pitch SP = M+1
// (the in-place FFT layout holds M values; the extra slot lives in the pitch pad).
template <typename C> __device__ __forceinline__ void stage_store(C* buf, int s, int k, int SP, C v) { buf[s * SP + k] = v; }
template <typename C> __device__ __forceinline__ C stage_load(const C* buf, int s, int k, int SP) { return buf[s * SP + k]; }

// ---------------------------------------------------------------------------
// Functor interface (F):
//   static constexpr int NR;                      // reduced doubles (0: none)
//   struct Ctx; static Ctx prep(const Desc<T>&);  // per-block constants
//   static bool skip(const Desc<T>&);             // whole-problem early exit
//   static void pixel(const Desc<T>&, const Ctx&, size_t i, T (&v)[NC], Acc<T> (&acc)[NR]);
//   static void finalize(const Desc<T>&, const double (&tot)[NR]);   // one thread
template <typename T, int NX, int NC, class F>
__global__ void __launch_bounds__(RowCfg<T, NX, NC>::NT) k_row_fwd(const Desc<T>* __restrict__ descs) {
    using Cfg = RowCfg<T, NX, NC>;
    using C = typename CT<T>::t;
    constexpr int M = Cfg::M, SP = Cfg::SP, ROWS = Cfg::ROWS, NT = Cfg::NT;
    const Desc<T>& d = descs[blockIdx.y];
    if (F::skip(d)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    T* rb = reinterpret_cast<T*>(smem_raw);
    const int y0 = blockIdx.x * ROWS;
    const typename F::Ctx ctx = F::prep(d);
    constexpr int NRA = F::NR > 0 ? F::NR : 1;
    Acc<T> acc[NRA];
#pragma unroll 4
    for (int t = threadIdx.x; t < ROWS * NX; t += NT) {
        const int row = t / NX, x = t % NX;
        const size_t pix = (size_t)(y0 + row) * NX + x;
        T v[NC];
        F::pixel(d, ctx, pix, v, &acc[0]);
#pragma unroll
        for (int c = 0; c < NC; ++c) rb[(size_t)(c * ROWS + row) * 2 * SP + x] = v[c];
    }
    if constexpr (F::NR > 0) {
        double vals[F::NR], tot[F::NR];
#pragma unroll
        for (int k = 0; k < F::NR; ++k) vals[k] = acc[k].get();
        if (reduce_last<F::NR, NT>(vals, d.part, &d.ctrl->counter, gridDim.x, tot) && threadIdx.x == 0)
            F::finalize(d, tot);
    }
    __syncthreads();
    fft_smem<T, M, Cfg::NSEQ, SP, NT, false>(buf, d.tw);
    // real-to-complex post-processing: X[k] = Xe[k] + W_N^k Xo[k], k = 0..M
    const C* twN = d.tw + NX;
    const size_t plane = (size_t)d.ny * d.wp;
    for (int t = threadIdx.x; t < Cfg::NSEQ * (M + 1); t += NT) {
        const int s = t / (M + 1), k = t % (M + 1);
        const int c = s / ROWS, row = s % ROWS;
        C zk = buf[s * SP + (k == M ? 0 : k)];
        C zm = buf[s * SP + (k == 0 ? 0 : M - k)];
        zm.y = -zm.y;
        C e = C{T(0.5) * (zk.x + zm.x), T(0.5) * (zk.y + zm.y)};
        C o = C{T(0.5) * (zk.y - zm.y), T(-0.5) * (zk.x - zm.x)};
        C X = cadd(e, cmul(twN[k], o));
        d.S[c * plane + (size_t)(y0 + row) * d.wp + k] = X;
    }
}

template <typename T, int NX, int NC, class F>
__global__ void __launch_bounds__(RowCfg<T, NX, NC>::NT) k_row_inv(const Desc<T>* __restrict__ descs) {
    using Cfg = RowCfg<T, NX, NC>;
    using C = typename CT<T>::t;
    constexpr int M = Cfg::M, SP = Cfg::SP, ROWS = Cfg::ROWS, NT = Cfg::NT;
    const Desc<T>& d = descs[blockIdx.y];
    if (F::skip(d)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    const T* rb = reinterpret_cast<const T*>(smem_raw);
    const int y0 = blockIdx.x * ROWS;
    const C* twN = d.tw + NX;
    const size_t plane = (size_t)d.ny * d.wp;
    // complex-to-real pre-processing: Z[k] = A + i B,
    //   A = X[k] + conj(X[M-k]),  B = (X[k] - conj(X[M-k])) e^{+2 pi i k/N}
    // (imaginary parts of X[0] and X[M] are dropped, as for a real inverse).
    // stage the half spectrum rows in shared memory first (independent loads), then combine
    for (int t = threadIdx.x; t < Cfg::NSEQ * (M + 1); t += NT) {
        const int s = t / (M + 1), k = t % (M + 1);
        const int c = s / ROWS, row = s % ROWS;
        stage_store(buf, s, k, SP, d.S[c * plane + (size_t)(y0 + row) * d.wp + k]);
    }
    __syncthreads();
    C z[(Cfg::NSEQ * M + NT - 1) / NT];
#pragma unroll
    for (int u = 0; u < (Cfg::NSEQ * M + NT - 1) / NT; ++u) {
        const int t = threadIdx.x + u * NT;
        if ((Cfg::NSEQ * M) % NT == 0 || t < Cfg::NSEQ * M) {
            const int s = t / M, k = t % M;
            C xk = stage_load<C>(buf, s, k, SP), xm = stage_load<C>(buf, s, M - k, SP);
            if (k == 0) { xk.y = T(0); xm.y = T(0); }
            xm.y = -xm.y;
            C A = cadd(xk, xm);
            C B = cmulc(csub(xk, xm), twN[k]);
            z[u] = C{A.x - B.y, A.y + B.x};
        }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < (Cfg::NSEQ * M + NT - 1) / NT; ++u) {
        const int t = threadIdx.x + u * NT;
        if ((Cfg::NSEQ * M) % NT == 0 || t < Cfg::NSEQ * M) buf[(t / M) * SP + t % M] = z[u];
    }
    __syncthreads();
    fft_smem<T, M, Cfg::NSEQ, SP, NT, true>(buf, d.tw);
    const typename F::Ctx ctx = F::prep(d);
    constexpr int NRA = F::NR > 0 ? F::NR : 1;
    Acc<T> acc[NRA];
#pragma unroll 4
    for (int t = threadIdx.x; t < ROWS * NX; t += NT) {
        const int row = t / NX, x = t % NX;
        const size_t pix = (size_t)(y0 + row) * NX + x;
        T v[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) v[c] = rb[(size_t)(c * ROWS + row) * 2 * SP + x];
        F::pixel(d, ctx, pix, v, &acc[0]);
    }
    if constexpr (F::NR > 0) {
        double vals[F::NR], tot[F::NR];
#pragma unroll
        for (int k = 0; k < F::NR; ++k) vals[k] = acc[k].get();
        if (reduce_last<F::NR, NT>(vals, d.part, &d.ctrl->counter, gridDim.x, tot) && threadIdx.x == 0)
            F::finalize(d, tot);
    }
}

// Column pass: CWE adjacent columns kx of the half spectrum, all NC planes.
// OP::apply(d, kx, ky, vals[NC]) multiplies one mode (normalisation included).
template <typename T, int NY, int NC, class OP>
__global__ void __launch_bounds__(ColCfg<T, NY, NC>::NT) k_col(const Desc<T>* __restrict__ descs) {
    using Cfg = ColCfg<T, NY, NC>;
    using C = typename CT<T>::t;
    constexpr int CW = Cfg::CWE, SP = Cfg::SP, NT = Cfg::NT;
    const Desc<T>& d = descs[blockIdx.y];
    if (OP::skip(d)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    const int kx0 = blockIdx.x * CW;
    const size_t plane = (size_t)d.ny * d.wp;
    constexpr int TOT = NC * NY * CW;
    constexpr int LPT = (TOT + NT - 1) / NT;   // elements per thread, loaded before any is stored
    {
        C tmp[LPT];
#pragma unroll
        for (int u = 0; u < LPT; ++u) {
            const int t = threadIdx.x + u * NT;
            if (TOT % NT == 0 || t < TOT) {
                const int j = t % CW, ky = (t / CW) % NY, c = t / (CW * NY);
                tmp[u] = d.S[c * plane + (size_t)ky * d.wp + kx0 + j];
            }
        }
#pragma unroll
        for (int u = 0; u < LPT; ++u) {
            const int t = threadIdx.x + u * NT;
            if (TOT % NT == 0 || t < TOT) {
                const int j = t % CW, ky = (t / CW) % NY, c = t / (CW * NY);
                buf[(c * CW + j) * SP + ky] = tmp[u];
            }
        }
    }
    __syncthreads();
    fft_smem<T, NY, Cfg::NSEQ, SP, NT, false>(buf, d.tw);
    for (int t = threadIdx.x; t < CW * NY; t += NT) {
        const int ky = t % NY, j = t / NY;
        C v[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) v[c] = buf[(c * CW + j) * SP + ky];
        OP::apply(d, kx0 + j, ky, v);
#pragma unroll
        for (int c = 0; c < NC; ++c) buf[(c * CW + j) * SP + ky] = v[c];
    }
    __syncthreads();
    fft_smem<T, NY, Cfg::NSEQ, SP, NT, true>(buf, d.tw);
#pragma unroll 4
    for (int t = threadIdx.x; t < TOT; t += NT) {
        const int j = t % CW, ky = (t / CW) % NY, c = t / (CW * NY);
        d.S[c * plane + (size_t)ky * d.wp + kx0 + j] = buf[(c * CW + j) * SP + ky];
    }
}

// ---------------------------------------------------------------------------
// mode multipliers
// Signed wavenumber index of row ky (numpy fftfreq order); Nyquist flagged.
__device__ __forceinline__ int signed_k(int k, int n) { return k < n / 2 ? k : k - n; }

// Compatibility projection Gamma(n) (Sec. 3.1.1), zero at q = 0 and on
// Nyquist modes; scaled by 1/(nx ny).
template <typename T>
__device__ __forceinline__ void gamma_apply(const Desc<T>& d, int kx, int ky, typename CT<T>::t (&v)[3]) {
    using C = typename CT<T>::t;
    const int M = d.nx / 2;
    if (kx > M || kx == M || ky == d.ny / 2 || (kx == 0 && ky == 0)) {
        v[0] = C{T(0), T(0)}; v[1] = v[0]; v[2] = v[0];
        return;
    }
    T qx = T(kx) * T(d.k.two_pi_over_Lx);
    T qy = T(signed_k(ky, d.ny)) * T(d.k.two_pi_over_Ly);
    T inv = T(1) / sqrt(qx * qx + qy * qy);
    T n1 = qx * inv, n2 = qy * inv;
    T sc = T(d.k.inv_n);
    C a = v[0], b = v[1], c = v[2];
    C s1{n1 * a.x + n2 * c.x, n1 * a.y + n2 * c.y};      // zeta n
    C s2{n1 * c.x + n2 * b.x, n1 * c.y + n2 * b.y};
    C t{n1 * s1.x + n2 * s2.x, n1 * s1.y + n2 * s2.y};   // n . zeta n
    T n11 = n1 * n1, n22 = n2 * n2, n12 = n1 * n2;
    v[0] = C{sc * (T(2) * n1 * s1.x - t.x * n11), sc * (T(2) * n1 * s1.y - t.y * n11)};
    v[1] = C{sc * (T(2) * n2 * s2.x - t.x * n22), sc * (T(2) * n2 * s2.y - t.y * n22)};
    v[2] = C{sc * (n1 * s2.x + n2 * s1.x - t.x * n12), sc * (n1 * s2.y + n2 * s1.y - t.y * n12)};
}

// Collocation Laplacian multiplier -|2 pi q|^2 / (nx ny) (Sec. 3.1.2).
template <typename T>
__device__ __forceinline__ void lap_apply(const Desc<T>& d, int kx, int ky, typename CT<T>::t (&v)[1]) {
    T qx = T(kx) * T(d.k.two_pi_over_Lx);
    T qy = T(signed_k(ky, d.ny)) * T(d.k.two_pi_over_Ly);
    if (ky == d.ny / 2) qy = T(d.ny / 2) * T(d.k.two_pi_over_Ly);
    T m = -(qx * qx + qy * qy) * T(d.k.inv_n);
    v[0].x *= m;
    v[0].y *= m;
}

}  // namespace pff
