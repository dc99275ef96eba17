// Row-forward kernels (per-pixel prologue + real FFT along x) for one precision (PFF_REAL).
#include "kernels.cuh"

namespace pff {

template <typename T>
void launch_row_fwd(int op, int nx, int ny, const Desc<T>* d, int np, cudaStream_t st) {
    switch (op) {
        case RF_NEWTON: PFF_SIZE_SWITCH(nx, (go_row_fwd<T, N_, 3, FNewtonIn<T>>(d, np, ny, st, FAM_ROW_FWD * 16 + op))); break;
        case RF_CG: PFF_SIZE_SWITCH(nx, (go_row_fwd<T, N_, 3, FCgIn<T>>(d, np, ny, st, FAM_ROW_FWD * 16 + op))); break;
        case RF_PHI: PFF_SIZE_SWITCH(nx, (go_row_fwd<T, N_, 1, FPhiIn<T>>(d, np, ny, st, FAM_ROW_FWD * 16 + op))); break;
        case RF_PF_A: PFF_SIZE_SWITCH(nx, (go_row_fwd<T, N_, 1, FPfA1<T>>(d, np, ny, st, FAM_ROW_FWD * 16 + op))); break;
        case RF_PF_B: PFF_SIZE_SWITCH(nx, (go_row_fwd<T, N_, 1, FPfVIn<T>>(d, np, ny, st, FAM_ROW_FWD * 16 + op))); break;
        case RF_COPY3: PFF_SIZE_SWITCH(nx, (go_row_fwd<T, N_, 3, FCopyIn<T, 3>>(d, np, ny, st, FAM_ROW_FWD * 16 + op))); break;
        case RF_PF_Z: PFF_SIZE_SWITCH(nx, (go_row_fwd<T, N_, 1, FPfZIn<T>>(d, np, ny, st, FAM_ROW_FWD * 16 + op))); break;
        case RF_COPY1: PFF_SIZE_SWITCH(nx, (go_row_fwd<T, N_, 1, FCopyIn<T, 1>>(d, np, ny, st, FAM_ROW_FWD * 16 + op))); break;
        default: break;
    }
}
template void launch_row_fwd<PFF_REAL>(int, int, int, const Desc<PFF_REAL>*, int, cudaStream_t);

}  // namespace pff
