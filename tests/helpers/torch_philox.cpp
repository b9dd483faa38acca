// Independent Philox4x32-10 reference for the tests: PyTorch's header-only at::philox_engine.
// Reads lines "k0 k1 c0 c1 c2 c3" (decimal) on stdin and prints the 4 output words of the block
// with that key and counter.  philox_engine(seed, subsequence, offset) puts the seed in the key,
// the offset in counter words 0-1 and the subsequence in counter words 2-3.
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdio>
#include <cstdint>

int main() {
    unsigned long long k0, k1, c0, c1, c2, c3;
    while (std::scanf("%llu %llu %llu %llu %llu %llu", &k0, &k1, &c0, &c1, &c2, &c3) == 6) {
        uint64_t seed = (uint64_t)k0 | ((uint64_t)k1 << 32);
        uint64_t subsequence = (uint64_t)c2 | ((uint64_t)c3 << 32);
        uint64_t offset = (uint64_t)c0 | ((uint64_t)c1 << 32);
        at::philox_engine eng(seed, subsequence, offset);
        uint32_t a = eng(), b = eng(), c = eng(), d = eng();
        std::printf("%u %u %u %u\n", a, b, c, d);
    }
    return 0;
}
