// Launcher of the lane walk (lanes.cuh) over the compacted frames of the
// two-phase global count.
#include "lanes.cuh"

namespace pvt {

// Every emitted compacted frame (A.emit, the count in *A.emit_count capped
// at A.emit_cap); walk statistics to slot FRAMES_SLOT.
__global__ void __launch_bounds__(32 * LANE_WPB, 2) k_lanes(CountArgs A)
{
    extern __shared__ __align__(16) unsigned char smem[];
    LaneWork *lw = reinterpret_cast<LaneWork *>(smem);
    unsigned *sh32 = reinterpret_cast<unsigned *>(lw + LANE_WPB);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned long long emitted = *(volatile unsigned long long *)A.emit_count;
    const unsigned nitems = (unsigned)min(emitted, (unsigned long long)A.emit_cap);
    if (blockIdx.x == 0 && threadIdx.x == 0) A.stats[3 + NCLASS + 1] = emitted;
    for (int i = threadIdx.x; i < HIST_H * HIST_P; i += blockDim.x) sh32[i] = 0;
    __syncthreads();
    lane_walk(lw[wid], sh32, A, lane, nitems, NCLASS);
    lane_hist_flush(sh32, A);
}


static pvt_status launch_lanes_kernel(pvt_dag *g, const CountArgs &A, int phase, cudaStream_t s)
{
    constexpr size_t smem = lane_smem_bytes();
    auto kern = k_lanes;
    PVT_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    PVT_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * LANE_WPB, smem));
    if (per_sm < 1) {
        set_error("lane walk kernel cannot be resident (shared memory)");
        return PVT_ECUDA;
    }
    const unsigned grid = (unsigned)(g->num_sms * per_sm);
    phase_begin(g, phase, s);
    kern<<<grid, 32 * LANE_WPB, smem, s>>>(A);
    PVT_CK(cudaGetLastError());
    phase_end(g, phase, s);
    return PVT_OK;
}

// Frame counters of the second phase: the emitted count is final on the device.
static __global__ void k_lanes_frames_init(uint32_t *qctl, const unsigned long long *emit_count, unsigned cap)
{
    for (int i = threadIdx.x; i < QCTL_WORDS; i += blockDim.x)
        qctl[i] = i == Q_OUT ? (unsigned)min(*emit_count, (unsigned long long)cap) : 0u;
}

// Ring queue of a lane launch in the buffers of slot `q` of the dag.
static pvt_status lane_ring(pvt_dag *g, CountArgs &A, int q, cudaStream_t s)
{
    pvt_status st;
    if ((st = grow(g->qframes[q], (size_t)SPLIT_QCAP * FRAME_WORDS, s)) != PVT_OK) return st;
    if ((st = grow(g->qready[q], (size_t)SPLIT_QCAP * 2, s)) != PVT_OK) return st;
    PVT_CK(cudaMemsetAsync(g->qready[q].p, 0, (size_t)SPLIT_QCAP * 2 * sizeof(uint32_t), s));
    A.qframes = g->qframes[q].p;
    A.qready = g->qready[q].p;
    A.qdone = g->qready[q].p + SPLIT_QCAP;
    A.qctl = g->qctl + QCTL_WORDS * q;
    A.qcap = SPLIT_QCAP;
    return PVT_OK;
}

pvt_status launch_lanes_frames(pvt_dag *g, const CountArgs &base, cudaStream_t s)
{
    CountArgs A = base;
    A.cls = NCLASS;
    pvt_status st = lane_ring(g, A, 0, s);
    if (st != PVT_OK) return st;
    k_lanes_frames_init<<<1, 128, 0, s>>>(A.qctl, A.emit_count, A.emit_cap);
    PVT_CK(cudaGetLastError());
    g->stats.launches += 2;
    return launch_lanes_kernel(g, A, PH_FRAMES, s);
}

}  // namespace pvt
