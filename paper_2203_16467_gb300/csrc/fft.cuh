// fft.cuh -- shared-memory batched FFTs and the three kernel shapes of a
// 2-D spectral operator F^-1 M F (Sec. 3.1: the DFT pair; the normalisation
// 1/(nx ny) is folded into the mode multiplier M):
//   k_row_fwd : per-pixel prologue -> real FFT along x  -> half spectrum S
//   k_col     : FFT along y -> mode multiplier (Gamma, -|2 pi q|^2 or the band
//               limit) -> inverse FFT along y (k_col512: register radix-8 stages
//               for 512-point FP32 columns)
//   k_row_inv : half spectrum -> real inverse FFT along x -> per-pixel epilogue (+ reductions)
// The kernels' bodies are per-item device functions (a row group, a column
// group) that the persistent solve shares.  FFTs are radix-8 Stockham passes
// (one radix-2 or radix-4 pass first when log2 of the length is not a multiple
// of 3), register staged and in place in shared memory with padded indices,
// with twiddles from FP64-accurate tables.
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

// Padded index of element e of a sequence in shared memory: one empty slot per
// 16 elements.  With this padding every read and write pattern of the mixed
// radix-8/4/2 Stockham passes below touches each 8-byte slot column at most
// twice per warp (the minimum for 8-byte elements).
__device__ __forceinline__ int pidx(int e) { return e + (e >> 4); }
constexpr int padded_len(int M) { return M + M / 16; }

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

// 8-point DFT in registers: two 4-point DFTs of the even and odd samples and
// the twiddles W8^k (W8 = exp(-+ 2 pi i / 8)).
template <typename C, bool INV>
__device__ __forceinline__ void dft8(C (&u)[8]) {
    using T = decltype(u[0].x);
    const T h = T(0.70710678118654752440);
    C e0 = u[0], e1 = u[2], e2 = u[4], e3 = u[6];
    C o0 = u[1], o1 = u[3], o2 = u[5], o3 = u[7];
    dft4<C, INV>(e0, e1, e2, e3);
    dft4<C, INV>(o0, o1, o2, o3);
    C t1, t2, t3;
    if (!INV) {
        t1 = C{h * (o1.x + o1.y), h * (o1.y - o1.x)};
        t2 = C{o2.y, -o2.x};
        t3 = C{h * (o3.y - o3.x), -h * (o3.x + o3.y)};
    } else {
        t1 = C{h * (o1.x - o1.y), h * (o1.x + o1.y)};
        t2 = C{-o2.y, o2.x};
        t3 = C{-h * (o3.x + o3.y), h * (o3.x - o3.y)};
    }
    u[0] = cadd(e0, o0); u[4] = csub(e0, o0);
    u[1] = cadd(e1, t1); u[5] = csub(e1, t1);
    u[2] = cadd(e2, t2); u[6] = csub(e2, t2);
    u[3] = cadd(e3, t3); u[7] = csub(e3, t3);
}

// One Stockham pass of radix R over sequences [s0, s0+G) of length M stored at
// buf[s*SP + pidx(j)]; p = product of the radices of the previous passes.
//   butterfly i in [0, M/R): k = i mod p; inputs x[i + r M/R]; twiddle
//   w^(r k) with w = exp(-+2 pi i/(p R)); outputs y[(i - k) R + k + r p].
// Twiddles: w^k, w^2k (and w^4k for radix 8) from the table, the rest as products.
// TWP: the twiddle table is stored with padded indices (pidx), as when staged in
// shared memory, so that the strided reads of a warp spread over the banks.
template <typename T, int M, int R, int G, int NSEQ, int SP, int NT, bool INV, bool TWP = false>
__device__ __forceinline__ void stockham_pass(typename CT<T>::t* buf, int s0, int p, const typename CT<T>::t* tw) {
    using C = typename CT<T>::t;
    constexpr int NBS = M / R;           // butterflies per sequence
    constexpr int NB = G * NBS;          // butterflies in the round
    constexpr int PER = (NB + NT - 1) / NT;
    C u[PER][8];
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        int b = threadIdx.x + j * NT;
        int s = s0 + b / NBS, i = b % NBS;
        if ((NB % NT == 0 || b < NB) && s < NSEQ) {
#pragma unroll
            for (int r = 0; r < R; ++r) u[j][r] = buf[s * SP + pidx(i + r * NBS)];
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        int b = threadIdx.x + j * NT;
        int s = s0 + b / NBS, i = b % NBS;
        if ((NB % NT == 0 || b < NB) && s < NSEQ) {
            const int k = i & (p - 1);
            if (p > 1) {
                const int idx = k * (M / (p * R));
                C w1 = tw[TWP ? pidx(idx) : idx];
                if (INV) w1.y = -w1.y;
                if (R == 2) {
                    u[j][1] = cmul(u[j][1], w1);
                } else {
                    C w2 = tw[TWP ? pidx(2 * idx) : 2 * idx];
                    if (INV) w2.y = -w2.y;
                    C w3 = cmul(w1, w2);
                    u[j][1] = cmul(u[j][1], w1);
                    u[j][2] = cmul(u[j][2], w2);
                    u[j][3] = cmul(u[j][3], w3);
                    if (R == 8) {
                        C w4 = tw[TWP ? pidx(4 * idx) : 4 * idx];
                        if (INV) w4.y = -w4.y;
                        u[j][4] = cmul(u[j][4], w4);
                        u[j][5] = cmul(u[j][5], cmul(w1, w4));
                        u[j][6] = cmul(u[j][6], cmul(w2, w4));
                        u[j][7] = cmul(u[j][7], cmul(w3, w4));
                    }
                }
            }
            if (R == 8) {
                dft8<C, INV>(u[j]);
            } else if (R == 4) {
                dft4<C, INV>(u[j][0], u[j][1], u[j][2], u[j][3]);
            } else {
                C a = u[j][0], c = u[j][1];
                u[j][0] = cadd(a, c);
                u[j][1] = csub(a, c);
            }
            const int o = (i - k) * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) buf[s * SP + pidx(o + r * p)] = u[j][r];
        }
    }
    __syncthreads();
}

// NSEQ in-place complex FFTs of length M (unnormalised; forward e^-, inverse e^+),
// radix-8 passes after one radix-2 or radix-4 pass when log2 M is not a multiple
// of 3.  Sequences are processed in rounds of G; each thread holds at most PER8
// radix-8 butterflies of a round in registers.
template <typename T, int M, int NSEQ, int SP, int NT, bool INV, bool TWP = false>
__device__ __forceinline__ void fft_smem(typename CT<T>::t* buf, const typename CT<T>::t* tw) {
    constexpr int LOG = ilog2(M);
    constexpr int PER8 = sizeof(T) == 4 ? 2 : 1;
    constexpr int G = cmax(1, cmin(NSEQ, (8 * NT * PER8) / M));   // sequences per round
    for (int s0 = 0; s0 < NSEQ; s0 += G) {
        int p = 1;
        if (LOG % 3 == 1) {
            stockham_pass<T, M, 2, G, NSEQ, SP, NT, INV, TWP>(buf, s0, 1, tw);
            p = 2;
        } else if (LOG % 3 == 2) {
            stockham_pass<T, M, 4, G, NSEQ, SP, NT, INV, TWP>(buf, s0, 1, tw);
            p = 4;
        }
        for (; p < M; p *= 8) stockham_pass<T, M, 8, G, NSEQ, SP, NT, INV, TWP>(buf, s0, p, tw);
    }
}

// cp.async: asynchronous global -> shared copies (no register staging)
// (PFF_L2_ONLY: translation units whose kernels read data written by other blocks of
// the same launch copy 8-byte elements with L2-only loads instead: cp.async.ca
// would go through L1, which is not coherent between SMs within a kernel.)
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
#ifdef PFF_L2_ONLY
    if constexpr (BYTES == 8) {
        *reinterpret_cast<unsigned long long*>(smem) = __ldcg(reinterpret_cast<const unsigned long long*>(gmem));
        return;
    }
#endif
    unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(gmem), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
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
    // FP32 forward passes: ask the register allocator for 8 resident 128-thread
    // blocks per SM (64 registers), so that enough loads are in flight, on the
    // sizes where the tangent of the mechanics pass fits without spilling; the
    // 512-point three-component pass takes 9 (56 registers, 8 bytes of spill:
    // measured 0.7 % faster in the concurrent-stream launch mode)
    static constexpr int MINB = (sizeof(T) == 4 && (NX == 128 || NX == 512 || NX == 1024))
                                    ? (NX == 512 && NC == 3 ? 9 : 8) * 128 / NT : 1;
    // FP32 512-point inverse passes: 7 resident blocks per SM (72 registers; 16-40 bytes of
    // spill in the update kernels), measured faster than 6 blocks at 80 registers and 5 at 96
    // when the one- and three-component passes of concurrent simulations share the SMs (8 at 64
    // registers spills 72 bytes and was slower)
    static constexpr int MINB_INV = (sizeof(T) == 4 && NX == 512) ? 7 : 1;
    static constexpr int SP = padded_len(M) + 2;            // pitch (complex): padded M values + slot for k = M
    static constexpr int NSEQ = NC * ROWS;
    // twiddles staged in shared memory: length-M FFT table (padded indices) + the
    // real-FFT factors exp(-2 pi i k / NX), k < M/2 (the split handles k and M - k together)
    static constexpr int TWF = padded_len(M);
    static constexpr int TWS = TWF + M / 2;
    static constexpr size_t SMEM = (size_t)(NSEQ * SP + TWS) * sizeof(typename CT<T>::t);
};

template <typename T, int NY, int NC>
struct ColCfg {
    static constexpr int CSZ = (int)sizeof(typename CT<T>::t);
    static constexpr int CWMIN = 32 / CSZ;                   // one 32-byte sector per row segment
    // one 32-byte sector per row segment: enough columns per block for full
    // sectors, and as many blocks as possible
    static constexpr int CWE = CWMIN;
    static constexpr int SP = ((padded_len(NY) + 7) / 16) * 16 + 8;   // pitch = 8 (mod 16) slots
    static constexpr int NSEQ = NC * CWE;
    static constexpr int NT = (NSEQ * NY >= 8192) ? 512 : (NSEQ * NY >= 2048 ? 256 : 128);
    // twiddles in shared memory when they fit next to the data (not for FP64 at 2048)
    static constexpr bool TW_SMEM = (size_t)(NSEQ * SP + padded_len(NY)) * CSZ <= 225 * 1024;
    static constexpr size_t SMEM = (size_t)(NSEQ * SP + (TW_SMEM ? padded_len(NY) : 0)) * CSZ;
};

constexpr int WP_ALIGN = 16;   // spectral row pitch multiple (largest column tile)

// Per-block mode constants in the storage precision (converted from FP64 once
// per thread, never per element: the FP64 pipe is narrow).
template <typename T>
struct ModeK {
    T cx, cy, inv_n;
    int nx, ny;
    const Consts* kc;       // the problem constants (read only by rarely used multipliers)
    T pre_a, pre_k;         // preconditioner (a_mean, 2 c ell^2), set by multipliers that need them
    ModeK() = default;
    __device__ __forceinline__ explicit ModeK(const Desc<T>& d)
        : cx(T(d.k.two_pi_over_Lx)), cy(T(d.k.two_pi_over_Ly)), inv_n(T(d.k.inv_n)), nx(d.nx), ny(d.ny), kc(&d.k) {}
};


// real value x of a real sequence stored as complex pairs z[n] = x[2n] + i x[2n+1]
__device__ __forceinline__ int ridx(int x) { return 2 * pidx(x >> 1) + (x & 1); }

// ---------------------------------------------------------------------------
// Functor interface (F):
//   static constexpr int NR;                      // reduced doubles (0: none)
//   struct Ctx; static Ctx prep(const Desc<T>&);  // per-block constants
//   static bool skip(const Desc<T>&);             // whole-problem early exit
//   static void pixel(const Desc<T>&, const Ctx&, size_t i, T (&v)[NC], Acc<T> (&acc)[NR]);
//   static void finalize(const Desc<T>&, const double (&tot)[NR]);   // one thread
#ifndef PFF_ROW_G
#define PFF_ROW_G 2
#endif
// Row-inverse passes issue the epilogue's pixel loads before staging and transforming the
// spectrum (they land during the FFT) when a thread handles at most this many pixels.
#ifndef PFF_INV_PREFETCH
#define PFF_INV_PREFETCH 8
#endif
template <class F, bool TWO> struct InOf { struct type {}; };
template <class F> struct InOf<F, true> { using type = typename F::In; };

// Row-forward pass of one row group y0 (ROWS rows): pixel prologue into the
// sequence buffer (accumulating F's reductions in acc) ...
template <typename T, int NX, int NC, class F>
__device__ __forceinline__ void row_fwd_pixels(const Desc<T>& d, const typename F::Ctx& ctx, int y0,
                                               typename CT<T>::t* buf, Acc<T>* acc) {
    using Cfg = RowCfg<T, NX, NC>;
    constexpr int SP = Cfg::SP, ROWS = Cfg::ROWS, NT = Cfg::NT;
    T* rb = reinterpret_cast<T*>(buf);
    if constexpr (HasIn<F>::value && (ROWS * NX) % NT == 0) {
        constexpr int PPT = ROWS * NX / NT;
        // pixels whose loads are in flight together: PFF_ROW_G, or as many as about 32
        // registers of loaded values allow (a power of two, so that it divides PPT)
        constexpr int WORDS = (int)((sizeof(typename F::In) + 3) / 4);
        constexpr int G = pow2floor(cmin(PPT, cmax(PFF_ROW_G, 32 / WORDS)));
#pragma unroll
        for (int j0 = 0; j0 < PPT; j0 += G) {
            typename F::In in[G];
#pragma unroll
            for (int j = 0; j < G; ++j) {
                const int t = threadIdx.x + (j0 + j) * NT;
                in[j] = F::load(d, ctx, (size_t)(y0 + t / NX) * NX + t % NX);
            }
#pragma unroll
            for (int j = 0; j < G; ++j) {
                const int t = threadIdx.x + (j0 + j) * NT;
                const int row = t / NX, x = t % NX;
                T v[NC];
                F::pixel(d, ctx, (size_t)(y0 + row) * NX + x, in[j], v, acc);
#pragma unroll
                for (int c = 0; c < NC; ++c) rb[(c * ROWS + row) * 2 * SP + ridx(x)] = v[c];
            }
        }
    } else {
#pragma unroll 4
        for (int t = threadIdx.x; t < ROWS * NX; t += NT) {
            const int row = t / NX, x = t % NX;
            const size_t pix = (unsigned)(y0 + row) * NX + x;
            T v[NC];
            pixel_one<F>(d, ctx, pix, v, acc);
#pragma unroll
            for (int c = 0; c < NC; ++c) rb[(c * ROWS + row) * 2 * SP + ridx(x)] = v[c];
        }
    }
}

// ... then (after a barrier) the real FFT along x and the half-spectrum store.
template <typename T, int NX, int NC>
__device__ __forceinline__ void row_fwd_fft_store(const Desc<T>& d, int y0, typename CT<T>::t* buf,
                                                  const typename CT<T>::t* tws) {
    using Cfg = RowCfg<T, NX, NC>;
    using C = typename CT<T>::t;
    constexpr int M = Cfg::M, SP = Cfg::SP, ROWS = Cfg::ROWS, NT = Cfg::NT;
    fft_smem<T, M, Cfg::NSEQ, SP, NT, false, true>(buf, tws);
    // real-to-complex post-processing of z = FFT(x[2n] + i x[2n+1]):
    //   X[k] = e + t,  e = (z[k] + conj z[M-k]) / 2,  t = W_N^k (z[k] - conj z[M-k]) / 2i,
    // and, from the same two values, X[M-k] = conj(e - t) (W_N^(M-k) = -conj W_N^k);
    // k = 0 gives X[0] and X[M], and its lane also writes the self-paired X[M/2] = conj z[M/2].
    constexpr int H = M / 2;
    const C* twN = tws + Cfg::TWF;
    const unsigned plane = (unsigned)d.ny * d.wp;   // 32-bit indices: < 2^32 elements
    for (int t = threadIdx.x; t < Cfg::NSEQ * H; t += NT) {
        const int s = t / H, k = t % H;
        const int c = s / ROWS, row = s % ROWS;
        C* out = d.S + (c * plane + (unsigned)(y0 + row) * d.wp);
        C zk = buf[s * SP + pidx(k)];
        C zm = buf[s * SP + pidx(k == 0 ? 0 : M - k)];
        zm.y = -zm.y;
        C e = C{T(0.5) * (zk.x + zm.x), T(0.5) * (zk.y + zm.y)};
        C o = C{T(0.5) * (zk.y - zm.y), T(-0.5) * (zk.x - zm.x)};
        C tk = cmul(twN[k], o);
        out[k] = cadd(e, tk);
        out[M - k] = C{e.x - tk.x, tk.y - e.y};
        if (k == 0) {
            C zh = buf[s * SP + pidx(H)];
            out[H] = C{zh.x, -zh.y};
        }
    }
}

// staged row twiddles: FFT table of length M at pidx(j), then exp(-2 pi i k / NX), k < M/2
template <typename T, int NX, int NC>
__device__ __forceinline__ void stage_row_twiddles(const Desc<T>& d, typename CT<T>::t* tws) {
    using Cfg = RowCfg<T, NX, NC>;
    using C = typename CT<T>::t;
    constexpr int M = Cfg::M;
    for (int t = threadIdx.x; t < M + M / 2; t += blockDim.x)
        cp_async<sizeof(C)>(t < M ? &tws[pidx(t)] : &tws[Cfg::TWF + (t - M)], t < M ? &d.tw[M + t] : &d.tw[NX + (t - M)]);
}

template <typename T, int NX, int NC, class F>
__device__ __forceinline__ void row_fwd_body(const Desc<T>* __restrict__ descs) {
    using Cfg = RowCfg<T, NX, NC>;
    using C = typename CT<T>::t;
    constexpr int NT = Cfg::NT;
    const Desc<T>& d = descs[blockIdx.y];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    C* tws = buf + Cfg::NSEQ * Cfg::SP;
    pdl_enter();
    typename F::Ctx ctx;
    if (block_prep<F>(d, ctx)) return;
    // twiddles are needed only after the pixel phase: staged after the skip test,
    // so that the blocks of a skipped problem return at once
    stage_row_twiddles<T, NX, NC>(d, tws);
    const int y0 = blockIdx.x * Cfg::ROWS;
    constexpr int NRA = F::NR > 0 ? F::NR : 1;
    Acc<T> acc[NRA];
    row_fwd_pixels<T, NX, NC, F>(d, ctx, y0, buf, &acc[0]);
    if constexpr (F::NR > 0) {
        double tot[F::NR];
        if (reduce_acc<F::NR, NT>(acc, d.part, &d.ctrl->counter, gridDim.x, tot) && threadIdx.x == 0)
            F::finalize(d, tot);
    }
    cp_async_wait_all();
    __syncthreads();
    row_fwd_fft_store<T, NX, NC>(d, y0, buf, tws);
}

// Each row kernel comes in two forms: with the register cap of its configuration (minimum
// resident blocks per SM; the FP32 sizes whose caps were chosen by measurement) and, suffix
// _u, without a minimum (the compiler's own choice: a minimum of one block is not the same as
// no bound to ptxas, which then takes more registers).
template <typename T, int NX, int NC, class F>
__global__ void __launch_bounds__(RowCfg<T, NX, NC>::NT, RowCfg<T, NX, NC>::MINB) k_row_fwd(const Desc<T>* __restrict__ descs) {
    row_fwd_body<T, NX, NC, F>(descs);
}
template <typename T, int NX, int NC, class F>
__global__ void __launch_bounds__(RowCfg<T, NX, NC>::NT) k_row_fwd_u(const Desc<T>* __restrict__ descs) {
    row_fwd_body<T, NX, NC, F>(descs);
}

// Row-inverse pass of one row group y0: the epilogue's pixel loads are issued
// first (they land during the staging and the FFT), the half-spectrum rows are
// staged, combined for the complex-to-real transform, transformed back along x,
// and the epilogue runs on the real values (accumulating F's reductions in acc).
template <typename T, int NX, int NC, class F>
__device__ __forceinline__ void row_inv_item(const Desc<T>& d, const typename F::Ctx& ctx, int y0,
                                             typename CT<T>::t* buf, const typename CT<T>::t* tws, Acc<T>* acc) {
    using Cfg = RowCfg<T, NX, NC>;
    using C = typename CT<T>::t;
    constexpr int M = Cfg::M, SP = Cfg::SP, ROWS = Cfg::ROWS, NT = Cfg::NT;
    const T* rb = reinterpret_cast<const T*>(buf);
    constexpr bool TWO = HasIn<F>::value && (ROWS * NX) % NT == 0 && ROWS * NX / NT <= PFF_INV_PREFETCH;
    constexpr int PPT = TWO ? ROWS * NX / NT : 1;
    using InT = typename InOf<F, TWO>::type;
    InT in[PPT];
    if constexpr (TWO) {
#pragma unroll
        for (int j = 0; j < PPT; ++j) {
            const int t = threadIdx.x + j * NT;
            in[j] = F::load(d, ctx, (size_t)((unsigned)(y0 + t / NX) * NX + t % NX));
        }
    }
    const C* twN = tws + Cfg::TWF;
    const unsigned plane = (unsigned)d.ny * d.wp;   // 32-bit indices: < 2^32 elements
    // complex-to-real pre-processing: Z[k] = A + i B,
    //   A = X[k] + conj(X[M-k]),  B = (X[k] - conj(X[M-k])) e^{+2 pi i k/N}
    // (imaginary parts of X[0] and X[M] are dropped, as for a real inverse); the same two
    // values give Z[M-k] = conj(A) + i conj(B), and Z[M/2] = 2 conj(X[M/2]) (k and M - k
    // together, k < M/2; the k = 0 lane forms Z[0] and Z[M/2]).
    // stage the half spectrum rows in shared memory (asynchronous copies), then combine
    for (int t = threadIdx.x; t < Cfg::NSEQ * (M + 1); t += NT) {
        const int s = t / (M + 1), k = t % (M + 1);
        const int c = s / ROWS, row = s % ROWS;
        cp_async<sizeof(C)>(&buf[s * SP + pidx(k)], &d.S[c * plane + (unsigned)(y0 + row) * d.wp + k]);
    }
    cp_async_wait_all();
    __syncthreads();
    constexpr int H = M / 2, NI = (Cfg::NSEQ * H + NT - 1) / NT;
    C z[NI][2];
#pragma unroll
    for (int u = 0; u < NI; ++u) {
        const int t = threadIdx.x + u * NT;
        if ((Cfg::NSEQ * H) % NT == 0 || t < Cfg::NSEQ * H) {
            const int s = t / H, k = t % H;
            C xk = buf[s * SP + pidx(k)], xm = buf[s * SP + pidx(M - k)];
            if (k == 0) { xk.y = T(0); xm.y = T(0); }
            xm.y = -xm.y;
            C A = cadd(xk, xm);
            C B = cmulc(csub(xk, xm), twN[k]);
            z[u][0] = C{A.x - B.y, A.y + B.x};
            z[u][1] = C{A.x + B.y, B.x - A.y};
            if (k == 0) {
                const C xh = buf[s * SP + pidx(H)];
                z[u][1] = C{T(2) * xh.x, T(-2) * xh.y};
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < NI; ++u) {
        const int t = threadIdx.x + u * NT;
        if ((Cfg::NSEQ * H) % NT == 0 || t < Cfg::NSEQ * H) {
            const int s = t / H, k = t % H;
            buf[s * SP + pidx(k)] = z[u][0];
            buf[s * SP + pidx(k == 0 ? H : M - k)] = z[u][1];
        }
    }
    __syncthreads();
    fft_smem<T, M, Cfg::NSEQ, SP, NT, true, true>(buf, tws);
    if constexpr (TWO) {
#pragma unroll
        for (int j = 0; j < PPT; ++j) {
            const int t = threadIdx.x + j * NT;
            const int row = t / NX, x = t % NX;
            T v[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) v[c] = rb[(c * ROWS + row) * 2 * SP + ridx(x)];
            F::pixel(d, ctx, (size_t)((unsigned)(y0 + row) * NX + x), in[j], v, acc);
        }
    } else {
        (void)in;
#pragma unroll 4
        for (int t = threadIdx.x; t < ROWS * NX; t += NT) {
            const int row = t / NX, x = t % NX;
            const size_t pix = (unsigned)(y0 + row) * NX + x;
            T v[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) v[c] = rb[(c * ROWS + row) * 2 * SP + ridx(x)];
            pixel_one<F>(d, ctx, pix, v, acc);
        }
    }
}

template <typename T, int NX, int NC, class F>
__device__ __forceinline__ void row_inv_body(const Desc<T>* __restrict__ descs) {
    using Cfg = RowCfg<T, NX, NC>;
    using C = typename CT<T>::t;
    constexpr int NT = Cfg::NT;
    const Desc<T>& d = descs[blockIdx.y];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    C* tws = buf + Cfg::NSEQ * Cfg::SP;
    pdl_enter();
    typename F::Ctx ctx;
    if (block_prep<F>(d, ctx)) return;
    stage_row_twiddles<T, NX, NC>(d, tws);
    constexpr int NRA = F::NR > 0 ? F::NR : 1;
    Acc<T> acc[NRA];
    row_inv_item<T, NX, NC, F>(d, ctx, blockIdx.x * Cfg::ROWS, buf, tws, &acc[0]);
    if constexpr (F::NR > 0) {
        double tot[F::NR];
        if (reduce_acc<F::NR, NT>(acc, d.part, &d.ctrl->counter, gridDim.x, tot) && threadIdx.x == 0)
            F::finalize(d, tot);
    }
}
template <typename T, int NX, int NC, class F>
__global__ void __launch_bounds__(RowCfg<T, NX, NC>::NT, RowCfg<T, NX, NC>::MINB_INV) k_row_inv(const Desc<T>* __restrict__ descs) {
    row_inv_body<T, NX, NC, F>(descs);
}
template <typename T, int NX, int NC, class F>
__global__ void __launch_bounds__(RowCfg<T, NX, NC>::NT) k_row_inv_u(const Desc<T>* __restrict__ descs) {
    row_inv_body<T, NX, NC, F>(descs);
}

// Column pass: CWE adjacent columns kx of the half spectrum, all NC planes.
// OP::apply(d, kx, ky, vals[NC]) multiplies one mode (normalisation included).
// column multipliers may read further per-problem constants into the ModeK (mode_prep)
template <class OP, class = void> struct HasModePrep { static constexpr bool value = false; };
template <class OP> struct HasModePrep<OP, decltype((void)&OP::template mode_prep<float>, void())> {
    static constexpr bool value = true;
};

// Column multipliers may also reduce over the modes they see (before multiplying):
// OP::NR values, OP::accum(mk, kx, ky, v, acc) per mode, OP::finalize(d, tot) once.
template <class OP, class = void> struct ColNR { static constexpr int value = 0; };
template <class OP> struct ColNR<OP, decltype((void)OP::NR, void())> { static constexpr int value = OP::NR; };

// skip test and mode constants of a column pass, evaluated once per block
template <typename T, class OP>
struct ColPrep {
    __device__ static bool skip(const Desc<T>& d) { return OP::skip(d); }
    __device__ static ModeK<T> prep(const Desc<T>& d) {
        ModeK<T> m(d);
        if constexpr (HasModePrep<OP>::value) OP::mode_prep(d, m);
        return m;
    }
};

template <typename T, int NY, int NC, class OP>
__global__ void __launch_bounds__(ColCfg<T, NY, NC>::NT) k_col(const Desc<T>* __restrict__ descs) {
    using Cfg = ColCfg<T, NY, NC>;
    using C = typename CT<T>::t;
    constexpr int CW = Cfg::CWE, SP = Cfg::SP, NT = Cfg::NT;
    const Desc<T>& d = descs[blockIdx.y];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    pdl_enter();
    ModeK<T> mk;
    if (block_prep<ColPrep<T, OP>>(d, mk)) return;
    const C* tw = d.tw + NY;
    if constexpr (Cfg::TW_SMEM) {
        C* tws = buf + Cfg::NSEQ * SP;
        for (int t = threadIdx.x; t < NY; t += NT) cp_async<sizeof(C)>(&tws[pidx(t)], &d.tw[NY + t]);
        tw = tws;
    }
    const int kx0 = blockIdx.x * CW;
    const unsigned plane = (unsigned)d.ny * d.wp;   // 32-bit indices: < 2^32 elements
    constexpr int TOT = NC * NY * CW;
    for (int t = threadIdx.x; t < TOT; t += NT) {
        const int j = t % CW, ky = (t / CW) % NY, c = t / (CW * NY);
        cp_async<sizeof(C)>(&buf[(c * CW + j) * SP + pidx(ky)], &d.S[c * plane + (unsigned)ky * d.wp + kx0 + j]);
    }
    cp_async_wait_all();
    __syncthreads();
    fft_smem<T, NY, Cfg::NSEQ, SP, NT, false, Cfg::TW_SMEM>(buf, tw);
    constexpr int NRA = ColNR<OP>::value > 0 ? ColNR<OP>::value : 1;
    Acc<T> acc[NRA];
    for (int t = threadIdx.x; t < CW * NY; t += NT) {
        const int ky = t % NY, j = t / NY;
        C v[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) v[c] = buf[(c * CW + j) * SP + pidx(ky)];
        if constexpr (ColNR<OP>::value > 0) OP::accum(mk, kx0 + j, ky, v, acc);
        OP::apply(mk, kx0 + j, ky, v);
#pragma unroll
        for (int c = 0; c < NC; ++c) buf[(c * CW + j) * SP + pidx(ky)] = v[c];
    }
    __syncthreads();
    fft_smem<T, NY, Cfg::NSEQ, SP, NT, true, Cfg::TW_SMEM>(buf, tw);
#pragma unroll 4
    for (int t = threadIdx.x; t < TOT; t += NT) {
        const int j = t % CW, ky = (t / CW) % NY, c = t / (CW * NY);
        d.S[c * plane + (unsigned)ky * d.wp + kx0 + j] = buf[(c * CW + j) * SP + pidx(ky)];
    }
    if constexpr (ColNR<OP>::value > 0) {
        double tot[ColNR<OP>::value];
        if (reduce_acc<ColNR<OP>::value, NT>(acc, d.part, &d.ctrl->counter, gridDim.x, tot) && threadIdx.x == 0)
            OP::finalize(d, tot);
    }
}

// ---------------------------------------------------------------------------
// Column pass for ny = 512 with register-resident radix-8 stages (512 = 8 x 8 x 8).
// Thread (column j, lane t) loads rows t + 64 m (m < 8) of every component
// straight into registers and runs the three radix-8 stages with two
// shared-memory exchanges:
//   stage 1: DFT8 over m, twiddle W512^(n0 k1)           (n0 = the lane's index)
//   stage 2: lane (k1, a): DFT8 over b of stage-1 values at n0 = a + 8 b, twiddle W64^(a c)
//   stage 3: lane (k1, c): DFT8 over a -> modes k1 + 8 c + 64 e, e < 8
// (k1 = t / 8, a or c = t % 8).  The mode multiplier acts on the NC components a
// lane holds; the inverse runs the same stages with lane index t' = k1 + 8 c (the
// lane holds modes t' + 64 e) and ends on rows t' + 64 e, stored straight from
// registers.  Exchange layouts (per component and column, stride COL512_XS = 8
// mod 16 complex slots): stage-1 value (k1, n0) at 72 k1 + n0 + n0/8, stage-2
// value (k1, a, c) at 72 k1 + 9 a + c; every access of a warp touches each
// bank pair at most twice (FP32).
constexpr int COL512_CW = 4;       // default columns per block (one 32-byte sector per row in FP32; 2 selectable)
constexpr int COL512_XS = 584;     // exchange slots per component and column

template <typename C, bool INV>
__device__ __forceinline__ void tw8(const C* tws, int base, C (&w)[8]) {
    // W512^(base r) for r < 8 from the entries for r = 1, 2, 4 (conjugated for the
    // inverse); the staged table is padded like the sequences (pidx), so that the
    // strided reads of a warp do not collide in the shared-memory banks
    C w1 = tws[pidx(base)], w2 = tws[pidx(2 * base)], w4 = tws[pidx(4 * base)];
    if (INV) { w1.y = -w1.y; w2.y = -w2.y; w4.y = -w4.y; }
    const C w3 = cmul(w1, w2);
    w[1] = w1; w[2] = w2; w[3] = w3; w[4] = w4;
    w[5] = cmul(w1, w4); w[6] = cmul(w2, w4); w[7] = cmul(w3, w4);
}

template <typename T, bool INV, int NC, int CW>
__device__ __forceinline__ void fft512_reg(typename CT<T>::t (&u)[NC][8], int n0, int t, typename CT<T>::t* xb,
                                           const typename CT<T>::t* tws) {
    using C = typename CT<T>::t;
    constexpr int CS = CW * COL512_XS;   // component stride
    C w[8];
    // stage 1
    tw8<C, INV>(tws, n0, w);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        dft8<C, INV>(u[c]);
#pragma unroll
        for (int r = 1; r < 8; ++r) u[c][r] = cmul(u[c][r], w[r]);
    }
    __syncthreads();   // earlier readers of xb are done
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int k1 = 0; k1 < 8; ++k1) xb[c * CS + 72 * k1 + n0 + (n0 >> 3)] = u[c][k1];
    __syncthreads();
    // stage 2
    const int k1 = t >> 3, a = t & 7;
    tw8<C, INV>(tws, 8 * a, w);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
#pragma unroll
        for (int b = 0; b < 8; ++b) u[c][b] = xb[c * CS + 72 * k1 + a + 9 * b];
        dft8<C, INV>(u[c]);
#pragma unroll
        for (int r = 1; r < 8; ++r) u[c][r] = cmul(u[c][r], w[r]);
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int cc = 0; cc < 8; ++cc) xb[c * CS + 72 * k1 + 9 * a + cc] = u[c][cc];
    __syncthreads();
    // stage 3 (lane (k1, c) with c = a)
#pragma unroll
    for (int c = 0; c < NC; ++c) {
#pragma unroll
        for (int aa = 0; aa < 8; ++aa) u[c][aa] = xb[c * CS + 72 * k1 + 9 * aa + a];
        dft8<C, INV>(u[c]);
    }
}

template <typename T, int NC, int CW = COL512_CW>
struct Col512Cfg {
    static constexpr int NT = 64 * CW;
    static constexpr size_t SMEM = (size_t)(padded_len(512) + NC * CW * COL512_XS) * sizeof(typename CT<T>::t);
};

// staged column twiddles: exp(-2 pi i k / 512) at pidx(k), k < 512
template <typename T>
__device__ __forceinline__ void stage_col512_twiddles(const Desc<T>& d, typename CT<T>::t* tws) {
    for (int i = threadIdx.x; i < 512; i += blockDim.x) cp_async<sizeof(typename CT<T>::t)>(&tws[pidx(i)], &d.tw[512 + i]);
}

// Column pass of the CW columns kx0.. of the half spectrum (64 CW threads).
template <typename T, int NC, class OP, int CW>
__device__ __forceinline__ void col512_item(const Desc<T>& d, const ModeK<T>& mk, int kx0, typename CT<T>::t* xb,
                                            const typename CT<T>::t* tws, Acc<T>* acc = nullptr) {
    using C = typename CT<T>::t;
    const int j = threadIdx.x % CW, t = threadIdx.x / CW;
    const int kx = kx0 + j;
    const unsigned plane = (unsigned)d.ny * d.wp;   // 32-bit indices: < 2^32 elements
    C u[NC][8];
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int m = 0; m < 8; ++m) u[c][m] = d.S[c * plane + (unsigned)(t + 64 * m) * d.wp + kx];
    cp_async_wait_all();   // staged twiddles (a no-op when the caller has waited already)
    __syncthreads();
    fft512_reg<T, false, NC, CW>(u, t, t, xb + j * COL512_XS, tws);
    const int k1 = t >> 3, cc = t & 7;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        C v[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) v[c] = u[c][e];
        if constexpr (ColNR<OP>::value > 0) OP::accum(mk, kx, k1 + 8 * cc + 64 * e, v, acc);
        OP::apply(mk, kx, k1 + 8 * cc + 64 * e, v);
#pragma unroll
        for (int c = 0; c < NC; ++c) u[c][e] = v[c];
    }
    const int tp = k1 + 8 * cc;
    fft512_reg<T, true, NC, CW>(u, tp, t, xb + j * COL512_XS, tws);
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int e = 0; e < 8; ++e) d.S[c * plane + (unsigned)(tp + 64 * e) * d.wp + kx] = u[c][e];
}

template <typename T, int NC, class OP, int CW = COL512_CW>
__global__ void __launch_bounds__(64 * CW) k_col512(const Desc<T>* __restrict__ descs) {
    using C = typename CT<T>::t;
    const Desc<T>& d = descs[blockIdx.y];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tws = reinterpret_cast<C*>(smem_raw);
    C* xb = tws + padded_len(512);
    pdl_enter();
    ModeK<T> mk;
    if (block_prep<ColPrep<T, OP>>(d, mk)) return;
    stage_col512_twiddles<T>(d, tws);   // waited for inside the item, after its loads are issued
    constexpr int NRA = ColNR<OP>::value > 0 ? ColNR<OP>::value : 1;
    Acc<T> acc[NRA];
    col512_item<T, NC, OP, CW>(d, mk, blockIdx.x * CW, xb, tws, acc);
    if constexpr (ColNR<OP>::value > 0) {
        double tot[ColNR<OP>::value];
        if (reduce_acc<ColNR<OP>::value, 64 * CW>(acc, d.part, &d.ctrl->counter, gridDim.x, tot) &&
            threadIdx.x == 0)
            OP::finalize(d, tot);
    }
}

// ---------------------------------------------------------------------------
// mode multipliers
// Signed wavenumber index of row ky (numpy fftfreq order); Nyquist flagged.
__device__ __forceinline__ int signed_k(int k, int n) { return k < n / 2 ? k : k - n; }

// Compatibility projection Gamma(n) (Sec. 3.1.1), zero at q = 0 and on
// Nyquist modes; scaled by 1/(nx ny).
template <typename T>
__device__ __forceinline__ void gamma_apply(const ModeK<T>& m, int kx, int ky, typename CT<T>::t (&v)[3]) {
    using C = typename CT<T>::t;
    const int M = m.nx / 2;
    if (kx >= M || ky == m.ny / 2 || (kx == 0 && ky == 0)) {
        v[0] = C{T(0), T(0)}; v[1] = v[0]; v[2] = v[0];
        return;
    }
    T qx = T(kx) * m.cx;
    T qy = T(signed_k(ky, m.ny)) * m.cy;
    T inv;
    if constexpr (sizeof(T) == 4) inv = rsqrtf(qx * qx + qy * qy);   // 2 ulp, one instruction
    else inv = T(1) / sqrt(qx * qx + qy * qy);
    T n1 = qx * inv, n2 = qy * inv;
    T sc = m.inv_n;
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
__device__ __forceinline__ void lap_apply(const ModeK<T>& m, int kx, int ky, typename CT<T>::t (&v)[1]) {
    T qx = T(kx) * m.cx;
    T qy = T(signed_k(ky, m.ny)) * m.cy;
    T f = -(qx * qx + qy * qy) * m.inv_n;
    v[0].x *= f;
    v[0].y *= f;
}

}  // namespace pff
