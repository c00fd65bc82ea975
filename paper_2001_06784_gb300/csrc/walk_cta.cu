// Launcher of the CTA-per-root walk (cta.cuh) for the out-degree classes
// above 128: one resident block per SM, as many warps as shared memory
// holds beside the root's rows.
#include "cta.cuh"

namespace pvt {

template <int NW>
static pvt_status launch_cta_nw(pvt_dag *g, CountArgs A, int cls, int dmax, cudaStream_t s)
{
    using Lay = CtaLayout<NW>;
    auto kern = k_cta<NW>;
    int optin = 0;
    PVT_CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, g->device));
    const size_t fixed = Lay::bytes(0, dmax);
    int warps = fixed < (size_t)optin ? (int)(((size_t)optin - fixed) / (sizeof(LaneWork) + sizeof(CtaWarp))) : 0;
    warps = std::min(warps, CTA_MAXW);
    if (warps < 1) {
        set_error("CTA walk: shared memory too small for out-degree " + std::to_string(dmax));
        return PVT_EINVAL;
    }
    const size_t smem = Lay::bytes(warps, dmax);
    PVT_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    PVT_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * warps, smem));
    if (per_sm < 1) {
        set_error("CTA walk kernel cannot be resident");
        return PVT_ECUDA;
    }
    const unsigned blocks = std::max(1u, std::min<unsigned>((unsigned)(g->num_sms * per_sm), A.nroots));
    pvt_status st =
        grow(g->gstack[cls], (size_t)blocks * warps * Lay::stack_words(dmax) + (size_t)blocks * Lay::gather_words(dmax), s);
    if (st != PVT_OK) return st;
    A.gstack = g->gstack[cls].p;
    phase_begin(g, 1 + cls, s);
    kern<<<blocks, 32 * warps, smem, s>>>(A, dmax);
    PVT_CK(cudaGetLastError());
    phase_end(g, 1 + cls, s);
    g->stats.launches++;
    return PVT_OK;
}

pvt_status launch_cta_class(pvt_dag *g, const CountArgs &base, int cls, cudaStream_t s)
{
    const unsigned cnt = (unsigned)g->wcnt[cls];
    if (cnt == 0) return PVT_OK;
    CountArgs A = base;
    A.roots = g->wroots + g->wstart[cls];
    A.nroots = cnt;
    A.qhead = g->d_q + cls;
    A.cls = cls;
    // rows and stacks sized by the largest out-degree the class can hold
    const int cap = 32 << (cls - 1);
    const int dmax = std::min(cap, (int)g->alpha);
    switch (cls) {
        case 4: return launch_cta_nw<8>(g, A, cls, dmax, s);
        case 5: return launch_cta_nw<16>(g, A, cls, dmax, s);
        case 6: return dmax <= 768 ? launch_cta_nw<24>(g, A, cls, dmax, s) : launch_cta_nw<32>(g, A, cls, dmax, s);
        default:
            set_error("CTA walk: only the out-degree classes above 128");
            return PVT_EINVAL;
    }
}

}  // namespace pvt
