// Host-only probe of the ML search's tensor-core table (ml_tc_word): prints the table of one
// stage as hex words, fragment tile by fragment tile.  Built and run by
// tests/test_ml_table_host.py; no GPU is touched.
//   ml_table_probe <L> <tauL_0> ... <tauL_{R-1}>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "ml_table.h"

int main(int argc, char** argv)
{
    if (argc < 3) return 2;
    const int L = atoi(argv[1]), R = argc - 2;
    std::vector<int32_t> tauL(R);
    for (int r = 0; r < R; ++r) tauL[r] = atoi(argv[2 + r]);
    const int KT = sfft::ml_tc_rp(R) / 4, MT = (L + 7) / 8;
    printf("%d %d\n", MT, KT);
    for (int mt = 0; mt < MT; ++mt)
        for (int kt = 0; kt < KT; ++kt)
            for (int h = 0; h < 2; ++h)
                for (int l = 0; l < 32; ++l)
                    for (int e = 0; e < 4; ++e)
                        printf("%08x\n", sfft::ml_tc_word(L, R, tauL.data(), mt, kt, h, l, e));
    return 0;
}
