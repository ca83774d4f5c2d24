// FP32 Legendre kernel variants (ring pairs per thread, maps per pass) for
// the autotuner; variant 0 of each family is the default.
#include "legendre_kernels.cuh"

namespace shtg {

#define SV(SP, NR, NM) &launch_synth_v<float, SP, NR, NM>
#define AV(SP, NR, NM) &launch_analysis_v<float, SP, NR, NM>

const Variants32 &variants32() {
    static const Variants32 V = {
        {4, 4, 4, 4},
        {{SV(0, 4, 2), SV(0, 4, 4), SV(0, 2, 4), SV(0, 8, 2)},
         {SV(2, 2, 2), SV(2, 2, 1), SV(2, 4, 1), SV(2, 1, 4)}},
        {{AV(0, 4, 2), AV(0, 8, 1), AV(0, 8, 2), AV(0, 6, 2)},
         {AV(2, 2, 2), AV(2, 4, 1), AV(2, 3, 2), AV(2, 4, 2)}},
        {{{4, 2}, {4, 4}, {2, 4}, {8, 2}},
         {{2, 2}, {2, 1}, {4, 1}, {1, 4}},
         {{4, 2}, {8, 1}, {8, 2}, {6, 2}},
         {{2, 2}, {4, 1}, {3, 2}, {4, 2}}}};
    return V;
}

}  // namespace shtg
