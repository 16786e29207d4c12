// Host-only probe of the bucketization layout (pfa_layout.h): lays out one stage and prints
// its axes and passes as one line of JSON.  Built and run by tests/test_layout_host.py; no
// GPU is touched.
//   layout_probe <B> <esz> <max_smem> <allow_tc> [max_tile]
#include <cstdio>
#include <cstdlib>

#include "pfa_layout.h"

int main(int argc, char** argv)
{
    if (argc < 5) return 2;
    sfft::StageDesc s{};
    s.B = atoi(argv[1]);
    s.L = 1;
    const size_t esz = (size_t)atoi(argv[2]);
    const int max_smem = atoi(argv[3]);
    const bool allow_tc = atoi(argv[4]) != 0;
    const long long max_tile = argc > 5 ? atoll(argv[5]) : 0;
    sfft::PassDesc p1{}, p2{};
    sfft::PassPlan l1, l2;
    int32_t cursor = 0;
    bool two_pass = false;
    const int64_t tile_target = esz == 8 ? 4096 : 2048;
    const bool ok = sfft::pfa_layout_stage(&s, esz, max_smem, tile_target, &p1, &p2, &l1, &l2,
                                           &cursor, &two_pass, max_tile, allow_tc);
    printf("{\"ok\": %d, \"two_pass\": %d, \"split\": %d, \"tw_total\": %d, \"smem1\": %zu, "
           "\"smem2\": %zu, \"axes\": [",
           ok ? 1 : 0, two_pass ? 1 : 0, s.split, cursor, l1.smem, l2.smem);
    for (int a = 0; ok && a < s.n_axes; ++a)
        printf("%s{\"P\": %d, \"pow2\": %d, \"S\": %d, \"tw_off\": %d, \"tc\": %d}", a ? ", " : "",
               s.ax[a].P, s.ax[a].pow2, s.ax[a].S, s.ax[a].tw_off, s.ax[a].tc);
    printf("]}\n");
    return 0;
}
