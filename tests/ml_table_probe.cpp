// Host-only probe of the ML search's tensor-core tables (ml_tc_word, ml_tc16_word): prints
// the table of one stage as hex words, fragment tile by fragment tile.  Built and run by
// tests/test_ml_table_host.py; no GPU is touched.
//   ml_table_probe tf32|f16 <L> <tauL_0> ... <tauL_{R-1}>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "ml_table.h"

int main(int argc, char** argv)
{
    if (argc < 4) return 2;
    const bool f16 = strcmp(argv[1], "f16") == 0;
    const int L = atoi(argv[2]), R = argc - 3;
    std::vector<int32_t> tauL(R);
    for (int r = 0; r < R; ++r) tauL[r] = atoi(argv[3 + r]);
    const int KT = f16 ? sfft::ml_tc16_ktiles(R) : sfft::ml_tc_rp(R) / 4, MT = (L + 7) / 8;
    printf("%d %d\n", MT, KT);
    for (int mt = 0; mt < MT; ++mt)
        for (int kt = 0; kt < KT; ++kt)
            for (int h = 0; h < 2; ++h)
                for (int l = 0; l < 32; ++l)
                    for (int e = 0; e < 4; ++e)
                        printf("%08x\n", f16 ? sfft::ml_tc16_word(L, R, tauL.data(), mt, kt, h, l, e)
                                             : sfft::ml_tc_word(L, R, tauL.data(), mt, kt, h, l, e));
    return 0;
}
