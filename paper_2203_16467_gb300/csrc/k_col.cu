// Column kernels (FFT along y, mode multiplier, inverse FFT along y) for one precision (PFF_REAL).
#include "kernels.cuh"

namespace pff {

template <typename T>
void launch_col(int op, int nx, int ny, int wp, const Desc<T>* d, int np, cudaStream_t st) {
    (void)wp;
    const int nm = nx / 2 + 1;   // columns kx = 0..nx/2 carry modes; the pitch's padding columns are left alone
    switch (op) {
        case CO_GAMMA_N: PFF_SIZE_SWITCH(ny, (go_col<T, N_, 3, FColGammaN>(d, np, nm, st, FAM_COL * 16 + op))); break;
        case CO_GAMMA_CG: PFF_SIZE_SWITCH(ny, (go_col<T, N_, 3, FColGammaCG>(d, np, nm, st, FAM_COL * 16 + op))); break;
        case CO_GAMMA_PLAIN: PFF_SIZE_SWITCH(ny, (go_col<T, N_, 3, FColGammaPlain>(d, np, nm, st, FAM_COL * 16 + op))); break;
        case CO_LAP_DF: PFF_SIZE_SWITCH(ny, (go_col<T, N_, 1, FColLapDF>(d, np, nm, st, FAM_COL * 16 + op))); break;
        case CO_LAP_PF: PFF_SIZE_SWITCH(ny, (go_col<T, N_, 1, FColLapPF>(d, np, nm, st, FAM_COL * 16 + op))); break;
        case CO_LAP_PLAIN: PFF_SIZE_SWITCH(ny, (go_col<T, N_, 1, FColLapPlain>(d, np, nm, st, FAM_COL * 16 + op))); break;
        case CO_LAP_PF_FULL: PFF_SIZE_SWITCH(ny, (go_col<T, N_, 1, FColLapPFFull>(d, np, nm, st, FAM_COL * 16 + op))); break;
        case CO_PRECOND: PFF_SIZE_SWITCH(ny, (go_col<T, N_, 1, FColPrecond>(d, np, nm, st, FAM_COL * 16 + op))); break;
        case CO_LAP_PFQ: PFF_SIZE_SWITCH(ny, (go_col<T, N_, 1, FColLapPFQ>(d, np, nm, st, FAM_COL * 16 + op))); break;
        case CO_LOWPASS: PFF_SIZE_SWITCH(ny, (go_col<T, N_, 1, FColLowPass>(d, np, nm, st, FAM_COL * 16 + op))); break;
        default: break;
    }
}
template void launch_col<PFF_REAL>(int, int, int, int, const Desc<PFF_REAL>*, int, cudaStream_t);

}  // namespace pff
