// Cell binning and spatial reorder (Sec. 2.2: O(N) cell search over cubic cells; the
// paper's per-cell linked lists become a counting sort into contiguous cell segments).
//
// Every kernel here is gated on sc->rebuild: when the integrator has not raised the flag
// the kernels return at once, so a captured step can always contain them.  All kernels
// use fixed grid-stride grids (a few blocks per SM) so that a skipped rebuild costs only
// a handful of empty launches.
//
// Chain: zero counts -> bin (key + histogram) -> exclusive scan -> scatter -> order each
// cell by id (canonical order: the sorted state depends only on positions and ids) ->
// gather into the alternate buffers (+ frame-relative FP32 copies) -> copy back.
#include "bbmd_internal.cuh"

namespace bbmd {

namespace {

constexpr int kThreads = 256;
#include "sort_bodies.cuh"

BBMD_ONE_AND_MANY(kThreads, k_zero, zero_body)
BBMD_ONE_AND_MANY(kThreads, k_bin, bin_body)
BBMD_ONE_AND_MANY(kScanThreads, k_scan_reduce, scan_reduce_body)
BBMD_ONE_AND_MANY(kScanThreads, k_scan_top, scan_top_body)
BBMD_ONE_AND_MANY(kScanThreads, k_scan_down, scan_down_body)
BBMD_ONE_AND_MANY(kThreads, k_scatter, scatter_body)
BBMD_ONE_AND_MANY(kThreads, k_cellsort, cellsort_body)
BBMD_ONE_AND_MANY(kThreads, k_gather, gather_body)
BBMD_ONE_AND_MANY(kThreads, k_copyback, copyback_body)

}  // namespace

int scan_grid(const DevSim& s) {
    const int nchunks = scan_chunks(s);
    return nchunks < 1 ? 1 : (nchunks < 1024 ? nchunks : 1024);
}

void launch_rebuild_chain(const DevSim& s, cudaStream_t st) {
    const int gscan = scan_grid(s);
    k_zero<<<s.grid_part, kThreads, 0, st>>>(s);
    k_bin<<<s.grid_part, kThreads, 0, st>>>(s);
    k_scan_reduce<<<gscan, kScanThreads, 0, st>>>(s);
    k_scan_top<<<1, kScanThreads, 0, st>>>(s);
    k_scan_down<<<gscan, kScanThreads, 0, st>>>(s);
    k_scatter<<<s.grid_part, kThreads, 0, st>>>(s);
    k_cellsort<<<s.grid_part, kThreads, 0, st>>>(s);
    k_gather<<<s.grid_part, kThreads, 0, st>>>(s);
    k_copyback<<<s.grid_part, kThreads, 0, st>>>(s);
}

void launch_rebuild_chain_many(const ManySims& part, const ManySims& scan, const ManySims& one,
                               int total_part, int total_scan, int nrep, cudaStream_t st) {
    k_zero_many<<<total_part, kThreads, 0, st>>>(part);
    k_bin_many<<<total_part, kThreads, 0, st>>>(part);
    k_scan_reduce_many<<<total_scan, kScanThreads, 0, st>>>(scan);
    k_scan_top_many<<<nrep, kScanThreads, 0, st>>>(one);
    k_scan_down_many<<<total_scan, kScanThreads, 0, st>>>(scan);
    k_scatter_many<<<total_part, kThreads, 0, st>>>(part);
    k_cellsort_many<<<total_part, kThreads, 0, st>>>(part);
    k_gather_many<<<total_part, kThreads, 0, st>>>(part);
    k_copyback_many<<<total_part, kThreads, 0, st>>>(part);
}

}  // namespace bbmd
