// Prints the library's tcgen05 descriptor encodings and tile offsets for the
// host test (tests/test_umma_desc.py), which checks them field by field.
#include <cstdio>

#include "umma_desc.h"

int main() {
    const unsigned starts[] = {0u, 16u, 1024u, 0x3FFF0u, 98304u + 256u};
    const unsigned lbos[] = {128u, 16u, 0x3FFF0u};
    const unsigned sbos[] = {1024u, 2048u, 16u};
    for (unsigned s : starts)
        for (unsigned l : lbos)
            for (unsigned b : sbos)
                std::printf("S %u %u %u %llu\n", s, l, b,
                            (unsigned long long)umma::smem_desc(s, l, b));
    const unsigned fm[][4] = {{2, 2, 128, 256}, {1, 1, 128, 64}, {0, 0, 64, 8}, {2, 2, 64, 128}};
    for (const auto& f : fm)
        std::printf("I %u %u %u %u %u\n", f[0], f[1], f[2], f[3],
                    umma::instr_desc(f[0], f[1], f[2], f[3]));
    for (unsigned r = 0; r < 256; r += 3)
        for (unsigned k = 0; k < 32; ++k)
            std::printf("O %u %u %u\n", r, k, umma::tf32_offset(r, k, 32));
    return 0;
}
