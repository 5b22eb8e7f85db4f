// Dispatch of the hop launches to the per-precision translation units
// (hop_f64_*.cu, hop_f32_*.cu, hop_f16_*.cu; kernels in hop_kernels.cuh) and
// the default launch configurations.
#include "dwf_internal.h"

namespace dwf {

template <int P, bool DAG>
cudaError_t hop_launch_pd(const HopArgs &a, int var, int NS, int SB, cudaStream_t st);
template <int P, bool DAG>
cudaError_t hop_batch_launch_pd(const HopArgs *tab, int nsys, const HopArgs &a0, int NS, int SB, cudaStream_t st);

// Defaults from the sweeps on 16^3x32, Ls 16 (GB300), chosen by the time to
// solution: FP16 variant 5 (0.206 s vs 0.210 s for variant 0), FP32 and FP64
// variant 0; one slice per thread (with the register caps above, the FP32 hop
// takes 106.3 us against 122.8 us with two slices).
int hop_default_variant(int prec) { return prec == DWF_F16 ? 5 : 0; }

int hop_default_ns(int prec, int Ls)
{
    (void)prec;
    (void)Ls;
    return 1;
}

int hop_default_sb(int prec, int Ls, int NS)
{
    (void)prec;
    const int LsN = Ls / NS;
    int sb = 128 / LsN;
    if (sb < 1) sb = 1;
    return sb;
}

cudaError_t launch_hop_batch(int prec, bool dag, const HopArgs *tab, int nsys, const HopArgs &a0, int NS, int SB,
                             cudaStream_t st)
{
    if (nsys < 1) return cudaSuccess;
    if (NS <= 0 || NS > 2 || (a0.Ls % NS) != 0) NS = hop_default_ns(prec, a0.Ls);
    if (SB <= 0) SB = hop_default_sb(prec, a0.Ls, NS);
    if ((a0.Ls / NS) * SB > 256) SB = 256 / (a0.Ls / NS);
    if (SB < 1) SB = 1;
    switch (prec) {
    case DWF_F64:
        return dag ? hop_batch_launch_pd<DWF_F64, true>(tab, nsys, a0, NS, SB, st)
                   : hop_batch_launch_pd<DWF_F64, false>(tab, nsys, a0, NS, SB, st);
    case DWF_F32:
        return dag ? hop_batch_launch_pd<DWF_F32, true>(tab, nsys, a0, NS, SB, st)
                   : hop_batch_launch_pd<DWF_F32, false>(tab, nsys, a0, NS, SB, st);
    case DWF_F16:
        return dag ? hop_batch_launch_pd<DWF_F16, true>(tab, nsys, a0, NS, SB, st)
                   : hop_batch_launch_pd<DWF_F16, false>(tab, nsys, a0, NS, SB, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_hop(int prec, bool dag, const HopArgs &a, int var, int NS, int SB, cudaStream_t st)
{
    if (var < 0 || var > 8 || var == 1 || var == 2) var = hop_default_variant(prec);
    if ((var == 7 || var == 8) && (prec == DWF_F64 || a.mixmode != 0 || a.Ls % 4 != 0)) {
        var = prec == DWF_F16 ? 5 : 0;   // variant 7 needs FP32/FP16 fields, dense mixing, Ls a multiple of 4
        SB = 0;
    }
    if (NS <= 0 || NS > 4 || NS == 3 || (a.Ls % NS) != 0 || (NS == 4 && var != 5)) NS = hop_default_ns(prec, a.Ls);
    if (var == 6 && (prec == DWF_F64 || a.mixmode != 0 || a.Ls > 32 || 32 % a.Ls != 0)) {
        var = prec == DWF_F16 ? 5 : 0;   // variant 6 needs FP32/FP16 fields, dense mixing, Ls dividing 32
        SB = 0;
        NS = hop_default_ns(prec, a.Ls);
    }
    if (var == 6) {   // one slice per thread; SB = warps per CTA (0: default)
        NS = 1;
        if (SB <= 0 || SB > 8) SB = 4;
        switch (prec) {
        case DWF_F32: return dag ? hop_launch_pd<DWF_F32, true>(a, 6, 1, SB, st) : hop_launch_pd<DWF_F32, false>(a, 6, 1, SB, st);
        case DWF_F16: return dag ? hop_launch_pd<DWF_F16, true>(a, 6, 1, SB, st) : hop_launch_pd<DWF_F16, false>(a, 6, 1, SB, st);
        default: var = 0; SB = 0; break;
        }
    }
    if (SB <= 0) SB = hop_default_sb(prec, a.Ls, NS);
    if ((a.Ls / NS) * SB > 256) SB = 256 / (a.Ls / NS);
    if (SB < 1) SB = 1;
    switch (prec) {
    case DWF_F64: return dag ? hop_launch_pd<DWF_F64, true>(a, var, NS, SB, st) : hop_launch_pd<DWF_F64, false>(a, var, NS, SB, st);
    case DWF_F32: return dag ? hop_launch_pd<DWF_F32, true>(a, var, NS, SB, st) : hop_launch_pd<DWF_F32, false>(a, var, NS, SB, st);
    case DWF_F16: return dag ? hop_launch_pd<DWF_F16, true>(a, var, NS, SB, st) : hop_launch_pd<DWF_F16, false>(a, var, NS, SB, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace dwf
