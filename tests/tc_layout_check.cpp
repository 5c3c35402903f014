// Host check of the tensor-core convolution's shared-memory descriptors
// (compiled by tests/test_tc_layout.py with a plain C++ compiler).  The
// descriptors are decoded here from the bit layout of the shared-memory
// matrix descriptor (start address, leading and stride byte offsets in
// 16-byte units, version bit 46, no swizzle), independently of the code
// that builds them, and every element an MMA would read is compared with
// the place the kernel's staging loop puts that element.
#define __host__
#define __device__
#include <cstdio>
#include <cstdint>
#include "../paper_1705_00614_gb300/csrc/swe_conv_tc.cuh"

using namespace swe;

static int fails = 0;

struct Desc {
    uint32_t start, lbo, sbo;
};

static Desc decode(uint64_t d) {
    const uint64_t known = 0x3FFFull | (0x3FFFull << 16) | (0x3FFFull << 32) | (7ull << 46) | (7ull << 49) |
                           (1ull << 52) | (7ull << 61);
    if ((d & ~known) != 0 || ((d >> 46) & 7) != 1 || ((d >> 49) & 7) != 0 || ((d >> 52) & 1) != 0 ||
        ((d >> 61) & 7) != 0) {
        std::printf("bad descriptor fields %llx\n", (unsigned long long)d);
        ++fails;
    }
    return Desc{(uint32_t)(d & 0x3FFF) << 4, (uint32_t)((d >> 16) & 0x3FFF) << 4, (uint32_t)((d >> 32) & 0x3FFF) << 4};
}

// K-major, no swizzle: 8 rows x 16 bytes per core matrix, rows 16 bytes apart
static uint32_t addr(const Desc& d, int row, int k) {
    return d.start + (uint32_t)(k / 8) * d.lbo + (uint32_t)(row / 8) * d.sbo + (uint32_t)(row % 8) * 16 +
           (uint32_t)(k % 8) * 2;
}

template <int CI, int CO>
static void check() {
    const uint32_t A0 = 0x400, W0 = A0 + conv_a_bytes<CI>() + 128;
    for (int tap = 0; tap < 9; ++tap) {
        const int dx = tap % 3;
        for (int s = 0; s < CI / 16; ++s)
            for (int slot = 0; slot < TC_RS; ++slot) {
                const Desc a = decode(smem_desc(A0 + conv_a_off<CI>(slot, dx, s), TC_A_LBO, TC_SBO));
                for (int k = 0; k < 16; ++k) {
                    const int c = 16 * s + k;
                    for (int m = 0; m < TCM; ++m) {
                        // output pixel m of the tile reads staged pixel m + dx of the slot's row
                        const uint32_t want = A0 + conv_a_stage<CI>(slot, c / 8, m + dx) + (uint32_t)(c % 8) * 2;
                        const uint32_t got = addr(a, m, k);
                        if (got != want || got < A0 || got + 2 > A0 + conv_a_bytes<CI>()) {
                            if (fails++ < 5)
                                std::printf("A CI=%d slot=%d dx=%d s=%d m=%d k=%d: %u vs %u\n", CI, slot, dx, s, m, k, got, want);
                        }
                    }
                }
            }
        for (int s = 0; s < CI / 16; ++s) {
            const Desc b = decode(smem_desc(W0 + conv_b_off<CI, CO>(tap, s), conv_b_lbo<CO>(), TC_SBO));
            for (int k = 0; k < 16; ++k) {
                const int c = 16 * s + k;  // input channel of this K element
                for (int o = 0; o < CO; ++o) {
                    const uint32_t want = W0 + conv_w_stage<CI, CO>(tap, c / 8, o) + (uint32_t)(c % 8) * 2;
                    const uint32_t got = addr(b, o, k);
                    if (got != want || got < W0 || got + 2 > W0 + conv_w_bytes<CI, CO>()) {
                        if (fails++ < 5) std::printf("B CI=%d CO=%d tap=%d s=%d o=%d k=%d: %u vs %u\n", CI, CO, tap, s, o, k, got, want);
                    }
                }
            }
        }
    }
    // staged pixels cover the tile and one pixel on each side
    if (TC_APAD < TCM + 2) ++fails;
    // instruction descriptor: F32 accumulator, BF16 A and B, K-major, N / 8, M / 16
    const uint32_t id = idesc_bf16_f32(TCM, CO);
    const uint32_t expect = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(CO / 8) << 17) | ((uint32_t)(TCM / 16) << 24);
    if (id != expect || ((id >> 17) & 0x3F) * 8 != (uint32_t)CO || ((id >> 24) & 0x1F) * 16 != (uint32_t)TCM) {
        std::printf("bad instruction descriptor %x\n", id);
        ++fails;
    }
    std::printf("CI=%d CO=%d checked\n", CI, CO);
}

int main() {
    check<16, 32>();
    check<32, 32>();
    check<32, 16>();
    std::printf(fails ? "FAIL %d\n" : "ok\n", fails);
    return fails ? 1 : 0;
}
