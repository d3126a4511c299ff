// Launch helpers for the pair kernel instantiations (one translation unit per
// precision and tangent count, so they compile in parallel).
#pragma once
#include "lcdm_kernels.cuh"

namespace lcdm {

typedef cudaError_t (*pairs_launch_fn)(const PairArgs&, int grid, int block, cudaStream_t);
typedef int (*pairs_occ_fn)(int block);

template <int PREC, int K, bool WT, bool WX>
cudaError_t launch_pairs(const PairArgs& a, int grid, int block, cudaStream_t s) {
    pairs_kernel<PREC, K, WT, WX><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}
template <int PREC, int K, bool WT, bool WX>
int occupancy_pairs(int block) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pairs_kernel<PREC, K, WT, WX>, block, 0) != cudaSuccess)
        return 0;
    return n;
}

// table entry for (WT, WX) = index (WT ? 2 : 0) + (WX ? 1 : 0)
struct PairsTable {
    pairs_launch_fn launch[4];
    pairs_occ_fn occ[4];
};

#define LCDM_DEFINE_TABLE(NAME, PREC, K)                                                     \
    PairsTable NAME() {                                                                      \
        PairsTable t;                                                                        \
        t.launch[0] = launch_pairs<PREC, K, false, false>;                                   \
        t.launch[1] = launch_pairs<PREC, K, false, true>;                                    \
        t.launch[2] = launch_pairs<PREC, K, true, false>;                                    \
        t.launch[3] = launch_pairs<PREC, K, true, true>;                                     \
        t.occ[0] = occupancy_pairs<PREC, K, false, false>;                                   \
        t.occ[1] = occupancy_pairs<PREC, K, false, true>;                                    \
        t.occ[2] = occupancy_pairs<PREC, K, true, false>;                                    \
        t.occ[3] = occupancy_pairs<PREC, K, true, true>;                                     \
        return t;                                                                            \
    }

PairsTable table_f64_k0();
PairsTable table_f64_k3();
PairsTable table_f64_k4();
PairsTable table_mix_k0();
PairsTable table_mix_k3();
PairsTable table_mix_k4();
PairsTable table_f64_k6();
// second pass of the deterministic reduction (defined with the other kernels)
cudaError_t launch_det_fixup(const PairArgs& a, int64_t nwarps, cudaStream_t s);
PairsTable table_mix_k6();

}  // namespace lcdm
