// FP64 Legendre kernel variants (ring pairs per thread, maps per pass) for
// the autotuner; variant 0 of each family is the default.
#include "legendre_kernels.cuh"

namespace shtg {

#define SV(SP, NR, NM) &launch_synth_v<double, SP, NR, NM>
#define AV(SP, NR, NM) &launch_analysis_v<double, SP, NR, NM>

const Variants64 &variants64() {
    static const Variants64 V = {
        {5, 4, 6, 4},
        {{SV(0, 2, 2), SV(0, 2, 4), SV(0, 1, 4), SV(0, 4, 2), SV(0, 4, 4)},
         {SV(2, 1, 2), SV(2, 1, 4), SV(2, 2, 2), SV(2, 2, 1)}},
        {{AV(0, 2, 1), AV(0, 4, 1), AV(0, 2, 2), AV(0, 8, 1), AV(0, 6, 1), AV(0, 4, 2)},
         {AV(2, 1, 1), AV(2, 2, 1), AV(2, 4, 1), AV(2, 3, 1)}},
        {{{2, 2}, {2, 4}, {1, 4}, {4, 2}, {4, 4}},
         {{1, 2}, {1, 4}, {2, 2}, {2, 1}},
         {{2, 1}, {4, 1}, {2, 2}, {8, 1}, {6, 1}, {4, 2}},
         {{1, 1}, {2, 1}, {4, 1}, {3, 1}}}};
    return V;
}

}  // namespace shtg
