// Dispatch of the hop launches to the per-precision translation units
// (hop_f64_*.cu, hop_f32_*.cu, hop_f16_*.cu; kernels in hop_kernels.cuh) and
// the default launch configurations.
#include "dwf_internal.h"

namespace dwf {

template <int P, bool DAG>
cudaError_t hop_launch_pd(const HopArgs &a, int var, int NS, int SB, cudaStream_t st);
template <int P, bool DAG>
cudaError_t hop_batch_launch_pd(const HopArgs *tab, int nsys, const HopArgs &a0, int NS, int SB, cudaStream_t st);

// Defaults from the sweeps on GB300 at 16^3x32 and 32^3x64, Ls 16: FP32 the
// warp-autonomous variant 9 (83.7 / 1446 us per hop against 102.4 / 1519 us for
// the direct variant 0; the whole FP32 CG iteration 475 / 7897 us against
// 586 / 8755 us), FP16 variant 5 (84.7 / 1183 us; variant 9: 87.8 / 1372 us),
// FP64 variant 0.  Variant 9 needs dense mixing and Ls dividing 32 (and a
// multiple of 4); otherwise the FP32 default is variant 0.
int hop_default_variant(int prec) { return prec == DWF_F16 ? 5 : (prec == DWF_F32 ? 9 : 0); }

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
    if (var < 0 || var > 10 || var == 1 || var == 2 || var == 6 || var == 8) var = hop_default_variant(prec);
    // variant 10 (variant 9 with the dense mixings on the tensor cores): FP32 fields, dense mixing,
    // Ls 8 or 16, no mixed y term; else variant 9
    if (var == 10) {
        if (prec == DWF_F32 && a.mixmode == 0 && a.ymode != 2 && (a.Ls == 8 || a.Ls == 16))
            return dag ? hop_launch_pd<DWF_F32, true>(a, 10, 0, 0, st) : hop_launch_pd<DWF_F32, false>(a, 10, 0, 0, st);
        var = 9;
        NS = 2;
        SB = 4;
    }
    // variants 7 and 9 need FP32/FP16 fields and dense mixing (9 also Ls dividing 32), else the default
    const bool v_ok = prec != DWF_F64 && a.mixmode == 0 && a.Ls % 4 == 0;
    const bool v9_ok = prec != DWF_F64 &&
                       ((a.mixmode == 0 && a.Ls % 4 == 0 && a.Ls <= 32 && 32 % a.Ls == 0) ||
                        (a.mixmode == 1 && (a.Ls == 8 || a.Ls == 16)));   // structured mixing: chains in registers
    if ((var == 7 && !v_ok) || (var == 9 && !v9_ok)) {
        var = prec == DWF_F16 ? 5 : 0;
        SB = 0;
        NS = 0;
    }
    if (var == 9) {   // SB = warps per CTA, NS = register budget (1: five CTAs per SM, 2: four)
        if (SB <= 0 || SB > 4) SB = 4;
        if (NS != 1) NS = 2;
        return prec == DWF_F32 ? (dag ? hop_launch_pd<DWF_F32, true>(a, 9, NS, SB, st)
                                      : hop_launch_pd<DWF_F32, false>(a, 9, NS, SB, st))
                               : (dag ? hop_launch_pd<DWF_F16, true>(a, 9, NS, SB, st)
                                      : hop_launch_pd<DWF_F16, false>(a, 9, NS, SB, st));
    }
    if (NS <= 0 || NS > 4 || NS == 3 || (a.Ls % NS) != 0 || (NS == 4 && var != 5) || var == 7)
        NS = hop_default_ns(prec, a.Ls);
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
