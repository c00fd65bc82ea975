// Walk kernels of the out-degree class with 32-word bitsets (vertex counts).
#include "walk.cuh"

namespace pvt {

template pvt_status launch_class<32, MODE_VERTEX, false>(pvt_dag *, const CountArgs &, int, cudaStream_t);

}  // namespace pvt
