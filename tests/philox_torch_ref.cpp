// Reads "c0 c1 c2 c3 k0 k1" (hex) lines on stdin and prints the Philox4x32-10
// block for each, computed by PyTorch's header-only at::philox_engine -- an
// implementation independent of the oracle, used to pin the oracle's Philox.
// The engine's seed is key0 | key1<<32, its subsequence counter words 2-3 and
// its offset counter words 0-1.
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdint>
#include <cstdio>

int main() {
    unsigned c[4], k[2];
    while (std::scanf("%x %x %x %x %x %x", &c[0], &c[1], &c[2], &c[3], &k[0], &k[1]) == 6) {
        uint64_t seed = (uint64_t)k[0] | ((uint64_t)k[1] << 32);
        uint64_t subseq = (uint64_t)c[2] | ((uint64_t)c[3] << 32);
        uint64_t offset = (uint64_t)c[0] | ((uint64_t)c[1] << 32);
        at::philox_engine eng(seed, subseq, offset);
        unsigned o0 = eng(), o1 = eng(), o2 = eng(), o3 = eng();
        std::printf("%08x %08x %08x %08x\n", o0, o1, o2, o3);
    }
    return 0;
}
