// Checks the integer-encoded float/double conversions of csrc/hx_convert.h against the host's own
// conversions (IEEE 754 round to nearest even): random encodings over all exponents, the binary32
// normal and subnormal boundaries, exact ties, and the specials.  Prints "ok <count>" or the
// first mismatch and exits non-zero.
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "hx_convert.h"

static uint64_t rng_state = 0x9e3779b97f4a7c15ull;
static uint64_t next()   // splitmix64
{
    uint64_t z = (rng_state += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

static long checked = 0;

static bool check_d2f(double x)
{
    const float ref = (float)x, got = hx::d2f_rn(x);
    ++checked;
    if (isnan(ref)) return isnan(got);
    if (hx::conv_bits32(ref) != hx::conv_bits32(got)) {
        printf("d2f_rn mismatch x=%a ref=%a got=%a\n", x, (double)ref, (double)got);
        return false;
    }
    float hi, lo;
    if (hx::d2f_split(x, hi, lo)) {
        const double err = fabs(((double)hi + (double)lo) - x), tail = fabs(x - (double)hi);
        if (hx::conv_bits32(hi) != hx::conv_bits32(ref) || err > 0x1p-23 * tail) {
            printf("d2f_split mismatch x=%a hi=%a lo=%a\n", x, (double)hi, (double)lo);
            return false;
        }
    } else if (x == 0.0 || (fabs(x) >= 0x1p-74 && fabs(x) < 0x1p100)) {
        printf("d2f_split refused x=%a\n", x);
        return false;
    }
    return true;
}

static bool check_f2d(float f)
{
    const double ref = (double)f, got = hx::f2d_exact(f);
    ++checked;
    if (isnan(f)) {
        if (!isnan(got) || (hx::conv_bits64(got) >> 29) != (hx::conv_bits64(ref) >> 29)) {
            printf("f2d NaN payload mismatch %08x\n", hx::conv_bits32(f));
            return false;
        }
        return true;
    }
    if (hx::conv_bits64(ref) != hx::conv_bits64(got)) {
        printf("f2d mismatch f=%a got=%a\n", (double)f, got);
        return false;
    }
    return true;
}

int main()
{
    // every binary64 exponent with random mantissas and signs
    for (uint64_t e = 0; e < 2048; ++e)
        for (int i = 0; i < 2000; ++i) {
            const uint64_t b = (next() & 0x800fffffffffffffull) | (e << 52);
            if (!check_d2f(hx::conv_from_bits64(b))) return 1;
        }
    // around the binary32 range: exponents 2^-155 .. 2^129, ties and near-ties of the dropped bits
    for (int E = -155; E <= 129; ++E)
        for (int i = 0; i < 20000; ++i) {
            uint64_t m = next() & 0xfffffffffffffull;
            const int kind = i % 4;
            const int drop = E >= -126 ? 29 : (E + 97 < -54 ? 52 : 29 + (-126 - E));
            const uint64_t dmask = drop >= 52 ? 0xfffffffffffffull : ((1ull << drop) - 1);
            if (kind == 1) m = (m & ~dmask) | (dmask >> 1) + 1;        // exact tie
            if (kind == 2) m = (m & ~dmask) | (dmask >> 1);            // just below the tie
            if (kind == 3) m = (m & ~dmask) | ((dmask >> 1) + 2);      // just above the tie
            const uint64_t b = ((next() & 1) << 63) | ((uint64_t)(E + 1023) << 52) | (m & 0xfffffffffffffull);
            if (!check_d2f(hx::conv_from_bits64(b))) return 1;
        }
    const double specials[] = {0.0, -0.0, INFINITY, -INFINITY, NAN, -NAN, 0x1p-149, 0x1p-150, 0x1.8p-150, 0x1p-151,
                               0x1.fffffep127, 0x1.ffffffp127, 0x1.fffffefffffffp127, 0x1p128, 0x1p-126,
                               0x1.fffffcp-127, 0x1p-1022, 0x1p-1074, 1.0, 1.0 + 0x1p-24, 1.0 + 0x1.8p-24};
    for (double x : specials)
        if (!check_d2f(x)) return 1;
    // binary32 -> binary64: all exponents (random mantissas), all subnormal mantissas below 2^16,
    // the top of the subnormals, specials
    for (uint32_t e = 0; e < 256; ++e)
        for (int i = 0; i < 20000; ++i) {
            const uint32_t b = ((uint32_t)next() & 0x807fffffu) | (e << 23);
            if (!check_f2d(hx::conv_from_bits32(b))) return 1;
        }
    for (uint32_t a = 0; a < 65536; ++a)
        if (!check_f2d(hx::conv_from_bits32(a)) || !check_f2d(hx::conv_from_bits32(0x80000000u | (0x7fffffu - a))))
            return 1;
    printf("ok %ld\n", checked);
    return 0;
}
