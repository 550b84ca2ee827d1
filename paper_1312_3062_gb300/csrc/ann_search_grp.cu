// ann_search_grp.cu -- the search kernels for indexes with the c2 group level
// (Algorithm 1, Sec. 4.2), instantiated in their own translation unit so that
// the kernels of indexes without groups keep their own register allocation and
// both compile in parallel.
#include "ann_search_dev.cuh"

namespace ann {

// the function's dynamic shared-memory limit is raised once to the opt-in
// maximum (a captured graph may hold nodes of one kernel with different sizes)
template <int DT, bool WIN>
static cudaError_t config_one(size_t smem, int threads, int *blocks_per_sm) {
    static bool raised = false;
    if (!raised) {
        int dev = 0, optin = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(search_kernel<DT, WIN, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
        if (e != cudaSuccess) return e;
        raised = true;
    }
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, search_kernel<DT, WIN, true>, threads, smem);
}

cudaError_t config_grouped(int dtype, bool win, size_t smem, int threads, int *blocks_per_sm) {
    if (dtype == ANN_U8)
        return win ? config_one<ANN_U8, true>(smem, threads, blocks_per_sm)
                   : config_one<ANN_U8, false>(smem, threads, blocks_per_sm);
    return win ? config_one<ANN_F32, true>(smem, threads, blocks_per_sm)
               : config_one<ANN_F32, false>(smem, threads, blocks_per_sm);
}

void launch_grouped(int dtype, bool win, dim3 grid, dim3 block, size_t smem, cudaStream_t s, const SearchArgs &A) {
    if (dtype == ANN_U8) {
        if (win) search_kernel<ANN_U8, true, true><<<grid, block, smem, s>>>(A);
        else search_kernel<ANN_U8, false, true><<<grid, block, smem, s>>>(A);
    } else {
        if (win) search_kernel<ANN_F32, true, true><<<grid, block, smem, s>>>(A);
        else search_kernel<ANN_F32, false, true><<<grid, block, smem, s>>>(A);
    }
}

}  // namespace ann
