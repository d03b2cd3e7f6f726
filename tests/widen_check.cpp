// Exhaustive check of the library's exact float -> double widening (an
// integer rebias of the IEEE-754 exponent, with the hardware conversion for
// subnormals, infinities and NaNs) against the compiler's conversion, bit
// for bit, over all 2^32 binary32 patterns.  Prints the number of
// mismatches.
#include <cstdio>
#include <cstring>
#include "../paper_2412_15518_gb300/csrc/common.cuh"

int main() {
    unsigned long long bad = 0;
    unsigned u = 0;
    do {
        float f;
        std::memcpy(&f, &u, 4);
        const double a = otfmm::widen(f), b = (double)f;
        unsigned long long x, y;
        std::memcpy(&x, &a, 8);
        std::memcpy(&y, &b, 8);
        if (x != y && bad++ < 5) std::printf("mismatch at 0x%08x\n", u);
    } while (++u != 0u);
    std::printf("%llu\n", bad);
    return bad != 0;
}
