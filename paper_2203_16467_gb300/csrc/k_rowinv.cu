// Row-inverse kernels (real inverse FFT along x + per-pixel epilogue) for one precision (PFF_REAL).
#include "kernels.cuh"

namespace pff {

template <typename T>
void launch_row_inv(int op, int nx, int ny, const Desc<T>* d, int np, cudaStream_t st) {
    switch (op) {
        case RI_NEWTON: PFF_SIZE_SWITCH(nx, (go_row_inv<T, N_, 3, FNewtonOut<T>>(d, np, ny, st, FAM_ROW_INV * 16 + op))); break;
        case RI_CG: PFF_SIZE_SWITCH(nx, (go_row_inv<T, N_, 3, FCgOut<T>>(d, np, ny, st, FAM_ROW_INV * 16 + op))); break;
        case RI_LAP: PFF_SIZE_SWITCH(nx, (go_row_inv<T, N_, 1, FLapOut<T>>(d, np, ny, st, FAM_ROW_INV * 16 + op))); break;
        case RI_ENERGY: PFF_SIZE_SWITCH(nx, (go_row_inv<T, N_, 1, FEnergyOut<T>>(d, np, ny, st, FAM_ROW_INV * 16 + op))); break;
        case RI_PF_A: PFF_SIZE_SWITCH(nx, (go_row_inv<T, N_, 1, FPfA3<T>>(d, np, ny, st, FAM_ROW_INV * 16 + op))); break;
        case RI_PF_B: PFF_SIZE_SWITCH(nx, (go_row_inv<T, N_, 1, FPfB3<T>>(d, np, ny, st, FAM_ROW_INV * 16 + op))); break;
        case RI_PF_Z: PFF_SIZE_SWITCH(nx, (go_row_inv<T, N_, 1, FPfZOut<T>>(d, np, ny, st, FAM_ROW_INV * 16 + op))); break;
        case RI_PF_AB: PFF_SIZE_SWITCH(nx, (go_row_inv<T, N_, 1, FPfA3B<T>>(d, np, ny, st, FAM_ROW_INV * 16 + op))); break;
        case RI_COPY3: PFF_SIZE_SWITCH(nx, (go_row_inv<T, N_, 3, FCopyOut<T, 3>>(d, np, ny, st, FAM_ROW_INV * 16 + op))); break;
        case RI_COPY1: PFF_SIZE_SWITCH(nx, (go_row_inv<T, N_, 1, FCopyOut<T, 1>>(d, np, ny, st, FAM_ROW_INV * 16 + op))); break;
        default: break;
    }
}
template void launch_row_inv<PFF_REAL>(int, int, int, const Desc<PFF_REAL>*, int, cudaStream_t);

}  // namespace pff
