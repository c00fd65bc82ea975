// Walk kernels of the out-degree class with 8-word bitsets.
#include "walk.cuh"

namespace pvt {

template pvt_status launch_class<8, MODE_GLOBAL, true>(pvt_dag *, const CountArgs &, int, cudaStream_t);
template pvt_status launch_class<8, MODE_VERTEX, false>(pvt_dag *, const CountArgs &, int, cudaStream_t);
template pvt_status launch_class<8, MODE_EDGE, false>(pvt_dag *, const CountArgs &, int, cudaStream_t);
template pvt_status launch_batch_class<8, MODE_GLOBAL>(const BatchGraph *, const uint64_t *, unsigned, unsigned *,
                                                    const unsigned long long *, int, unsigned *, unsigned long long *,
                                                    int, cudaStream_t);
template pvt_status launch_batch_class<8, MODE_VERTEX>(const BatchGraph *, const uint64_t *, unsigned, unsigned *,
                                                    const unsigned long long *, int, unsigned *, unsigned long long *,
                                                    int, cudaStream_t);
template pvt_status launch_batch_class<8, MODE_EDGE>(const BatchGraph *, const uint64_t *, unsigned, unsigned *,
                                                    const unsigned long long *, int, unsigned *, unsigned long long *,
                                                    int, cudaStream_t);

}  // namespace pvt
