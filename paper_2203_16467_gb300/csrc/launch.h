// launch.h -- host-side entry points of the kernel translation units.
#pragma once
#include <cuda_runtime.h>

namespace pff {

template <typename T> struct Desc;

enum RowFwdOp { RF_NEWTON, RF_CG, RF_PHI, RF_PF_A, RF_PF_B, RF_COPY3, RF_COPY1, RF_PF_Z };
enum RowInvOp { RI_NEWTON, RI_CG, RI_LAP, RI_ENERGY, RI_PF_A, RI_PF_B, RI_COPY3, RI_COPY1, RI_PF_Z, RI_PF_AB };
enum ColOp { CO_GAMMA_N, CO_GAMMA_CG, CO_GAMMA_PLAIN, CO_LAP_DF, CO_LAP_PF, CO_LAP_PLAIN, CO_LAP_PF_FULL, CO_LOWPASS, CO_PRECOND,
             CO_LAP_PFQ };
enum ElemOp { EL_FOLD, EL_PF_INIT, EL_POST, EL_DF, EL_CONSTITUTIVE, EL_STATE, EL_DRIVING, EL_FLAGS,
              EL_SAVE_CON, EL_SAVE_PHI, EL_RESTORE_PHI, EL_PF_B };

template <typename T> void launch_row_fwd(int op, int nx, int ny, const Desc<T>* d, int np, cudaStream_t st);
template <typename T> void launch_row_inv(int op, int nx, int ny, const Desc<T>* d, int np, cudaStream_t st);
template <typename T> void launch_col(int op, int nx, int ny, int wp, const Desc<T>* d, int np, cudaStream_t st);
template <typename T> void launch_elem(int op, int nx, int ny, const Desc<T>* d, int np, cudaStream_t st);
template <typename T> void launch_step_begin(const Desc<T>* d, int np, cudaStream_t st);
template <typename T> void launch_gather(const Desc<T>* d, int np, int* flags, void* ctrl_out, cudaStream_t st);
// sets the graph condition h to 1 when some problem of the group evaluates J v
// explicitly in this BCCG iteration (its pf_full is set and it has not stopped)
template <typename T> void launch_pf_cond(const Desc<T>* d, int np, cudaGraphConditionalHandle h, cudaStream_t st);
// the whole mechanics solve of np FP32 512 x 512 problems, one thread-block cluster each (k_cluster.cu)
bool mech_cluster_supported();
cudaError_t launch_mech_cluster(const Desc<float>* d, int np, cudaStream_t st);
void launch_convert_d2f(float* dst, const double* src, size_t n, cudaStream_t st);
void launch_convert_f2d(double* dst, const float* src, size_t n, cudaStream_t st);

}  // namespace pff
