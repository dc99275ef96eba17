// Elementwise kernels, the driving-force maximum and state resets for one precision (PFF_REAL).
#include "kernels.cuh"

namespace pff {

template <typename T, class F>
static void go_elem(int nx, int ny, const Desc<T>* d, int np, cudaStream_t st) {
    launch_pdl<T>(k_elem<T, F>, dim3(elem_blocks(nx, ny, np), np), dim3(EL_NT), 0, st, d);
    count_launch();
}

template <typename T>
void launch_elem(int op, int nx, int ny, const Desc<T>* d, int np, cudaStream_t st) {
    const bool tm = timing_on();
    if (tm) timing_begin(FAM_ELEM * 16 + op, st);
    switch (op) {
        case EL_FOLD: go_elem<T, FFold<T>>(nx, ny, d, np, st); break;
        case EL_PF_INIT: go_elem<T, FPfInit<T>>(nx, ny, d, np, st); break;
        case EL_POST: go_elem<T, FPost<T>>(nx, ny, d, np, st); break;
        case EL_DF:
            k_df<T><<<dim3(elem_blocks(nx, ny, np), np), EL_NT, 0, st>>>(d);
            count_launch();
            break;
        case EL_CONSTITUTIVE: go_elem<T, FConstitutive<T>>(nx, ny, d, np, st); break;
        case EL_STATE: go_elem<T, FStateFields<T>>(nx, ny, d, np, st); break;
        case EL_DRIVING: go_elem<T, FDrivingField<T>>(nx, ny, d, np, st); break;
        case EL_FLAGS: go_elem<T, FFlagsField<T>>(nx, ny, d, np, st); break;
        case EL_SAVE_CON: go_elem<T, FAux<T, 0>>(nx, ny, d, np, st); break;
        case EL_SAVE_PHI: go_elem<T, FAux<T, 1>>(nx, ny, d, np, st); break;
        case EL_RESTORE_PHI: go_elem<T, FAux<T, 2>>(nx, ny, d, np, st); break;
        case EL_PF_B: go_elem<T, FPfB1<T>>(nx, ny, d, np, st); break;
        default: break;
    }
    if (tm) timing_end(FAM_ELEM * 16 + op, st);
}
template void launch_elem<PFF_REAL>(int, int, int, const Desc<PFF_REAL>*, int, cudaStream_t);

template <typename T>
void launch_step_begin(const Desc<T>* d, int np, cudaStream_t st) {
    k_step_begin<T><<<(np + 127) / 128, 128, 0, st>>>(d, np);
    count_launch();
}
template void launch_step_begin<PFF_REAL>(const Desc<PFF_REAL>*, int, cudaStream_t);

// flags of every problem, and a contiguous copy of every control block
template <typename T>
__global__ void k_gather_all(const Desc<T>* __restrict__ descs, int np, int* flags, Ctrl* out) {
    int j = blockIdx.x;
    if (j >= np) return;
    const Ctrl* c = descs[j].ctrl;
    if (out) {
        const int* src = reinterpret_cast<const int*>(c);
        int* dst = reinterpret_cast<int*>(out + j);
        for (int w = threadIdx.x; w < (int)(sizeof(Ctrl) / sizeof(int)); w += blockDim.x) dst[w] = __ldcg(src + w);
    }
    if (threadIdx.x == 0 && flags)
        flags[j] = (__ldcg(&c->cg_b) ? 1 : 0) | (__ldcg(&c->nd_a) ? 2 : 0) | (__ldcg(&c->pf_b) ? 4 : 0);
}

template <typename T>
void launch_gather(const Desc<T>* d, int np, int* flags, void* ctrl_out, cudaStream_t st) {
    k_gather_all<T><<<np, 64, 0, st>>>(d, np, flags, reinterpret_cast<Ctrl*>(ctrl_out));
    count_launch();
}
template void launch_gather<PFF_REAL>(const Desc<PFF_REAL>*, int, int*, void*, cudaStream_t);

template <typename T>
__global__ void k_pf_cond(const Desc<T>* __restrict__ descs, int np, cudaGraphConditionalHandle h) {
    int any = 0;
    for (int j = threadIdx.x; j < np; j += blockDim.x) {
        const Ctrl* c = descs[j].ctrl;
        any |= (!__ldcg(&c->pf_a) && __ldcg(&c->pf_full)) ? 1 : 0;
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) cudaGraphSetConditional(h, any ? 1u : 0u);
}

template <typename T>
void launch_pf_cond(const Desc<T>* d, int np, cudaGraphConditionalHandle h, cudaStream_t st) {
    k_pf_cond<T><<<1, 64, 0, st>>>(d, np, h);
    count_launch();
}
template void launch_pf_cond<PFF_REAL>(const Desc<PFF_REAL>*, int, cudaGraphConditionalHandle, cudaStream_t);

}  // namespace pff
