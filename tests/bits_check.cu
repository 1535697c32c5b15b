// Host driver for the bit-pattern conversions of csrc/bits.cuh (compiled by
// nvcc for the host only; tests/test_bits_host.py feeds it and checks the
// answers against exact arithmetic).  One request per line on stdin:
//   S <double bits, hex>            -> hi, lo float bits of split_f32
//   Q <double bits, hex> <levels>   -> quantise_unit
//   F <double bits, hex> <E>        -> fixed_from_double, 128-bit two's complement hex
//   T <128-bit two's complement hex> -> fixed_to_double_trunc, double bits
#include <stdio.h>
#include <string.h>

#include "bits.cuh"

int main()
{
    char op[4], a[64];
    while (scanf("%3s %63s", op, a) == 2) {
        if (op[0] == 'T') {
            unsigned long long hi = 0, lo = 0;
            char h[17] = {0};
            memcpy(h, a, 16);
            sscanf(h, "%llx", &hi);
            sscanf(a + 16, "%llx", &lo);
            const __int128 v = (__int128)(((unsigned __int128)hi << 64) | lo);
            printf("%016llx\n", hts::bits_of(hts::fixed_to_double_trunc(v)));
            continue;
        }
        unsigned long long xb = 0;
        sscanf(a, "%llx", &xb);
        const double x = hts::double_of(xb);
        if (op[0] == 'S') {
            float hi, lo;
            hts::split_f32(x, hi, lo);
            unsigned hb, lb;
            memcpy(&hb, &hi, 4);
            memcpy(&lb, &lo, 4);
            printf("%08x %08x\n", hb, lb);
        } else {
            int k = 0;
            if (scanf("%d", &k) != 1) return 1;
            if (op[0] == 'Q') {
                printf("%llu\n", (unsigned long long)hts::quantise_unit(x, k));
            } else {
                const unsigned __int128 u = (unsigned __int128)hts::fixed_from_double(x, k);
                printf("%016llx%016llx\n", (unsigned long long)(u >> 64), (unsigned long long)u);
            }
        }
    }
    return 0;
}
