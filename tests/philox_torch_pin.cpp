// Independent Philox4x32-10 for pinning the oracle: PyTorch's header-only
// at::philox_engine.  Reads lines "k0 k1 c0 c1 c2 c3" from stdin and prints
// the four output words of Philox4x32-10(counter=(c0,c1,c2,c3), key=(k0,k1)).
#include <ATen/core/PhiloxRNGEngine.h>
#include <cinttypes>
#include <cstdio>

int main()
{
    unsigned long v[6];
    while (std::scanf("%lu %lu %lu %lu %lu %lu", &v[0], &v[1], &v[2], &v[3], &v[4], &v[5]) == 6) {
        uint64_t seed = (uint64_t)v[0] | ((uint64_t)v[1] << 32);
        uint64_t offset = (uint64_t)v[2] | ((uint64_t)v[3] << 32);
        uint64_t subsequence = (uint64_t)v[4] | ((uint64_t)v[5] << 32);
        at::philox_engine e(seed, subsequence, offset);
        uint32_t a = e(), b = e(), c = e(), d = e();
        std::printf("%u %u %u %u\n", a, b, c, d);
    }
    return 0;
}
