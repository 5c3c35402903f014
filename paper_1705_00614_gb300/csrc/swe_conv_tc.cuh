// Shared-memory layout of the tensor-core (tcgen05) 3x3 convolution and the
// matrix descriptors its MMAs use.  Host-and-device code, so the layout can
// be checked on the host (the descriptors are decoded there and every
// element they address is compared with the intended one).
//
// A tile is TCM = 128 consecutive output pixels of one image row (the MMA's
// M).  Input rows stream through a ring of TC_RS row slots; per slot, channel
// chunk kc (8 channels = 16 bytes) and pixel p (130: the tile plus one pixel
// on each side) the shared array holds 16 bytes at
// ((slot * NKC + kc) * TC_APAD + p) * 16 (one TMA box of 130 x 16 bytes per
// slot and chunk).  With no swizzling the MMA reads K-major 8 x 16-byte core
// matrices: 8 consecutive pixels of one chunk are 128 contiguous bytes (the
// stride between 8-row groups, SBO = 128), and the next chunk along K is
// TC_APAD * 16 bytes further (LBO).  The operand of tap (dy, dx) is the slot
// of input row i + dy - 1, started dx pixels later.  Weights are held as
// [tap][kc][o][8 channels]: SBO 128, LBO = CO * 16.
#pragma once

#include <stdint.h>

namespace swe {

constexpr int TCM = 128;      // output pixels per tile (MMA M)
constexpr int TC_APAD = 136;  // shared rows per (row slot, channel chunk); >= TCM + 2
constexpr int TC_RS = 6;      // row slots: 3 rows per tile, two tiles in flight, one row loading
constexpr uint32_t TC_SBO = 128;
constexpr uint32_t TC_A_LBO = TC_APAD * 16;

template <int CI>
__host__ __device__ constexpr uint32_t conv_a_bytes() {
    return (uint32_t)TC_RS * (CI / 8) * TC_APAD * 16;
}
template <int CI, int CO>
__host__ __device__ constexpr uint32_t conv_w_bytes() {
    return 9u * (CI / 8) * CO * 16;
}
// Where 16 bytes (8 channels) are staged: row slot, channel chunk kc, pixel
// p of the tile's row plus halo; weights of tap t, chunk kc, output channel o.
template <int CI>
__host__ __device__ constexpr uint32_t conv_a_stage(int slot, int kc, int p) {
    return (uint32_t)(((slot * (CI / 8) + kc) * TC_APAD + p) * 16);
}
template <int CI, int CO>
__host__ __device__ constexpr uint32_t conv_w_stage(int tap, int kc, int o) {
    return (uint32_t)(((tap * (CI / 8) + kc) * CO + o) * 16);
}
// Offset of the A operand of a tap whose input row sits in `slot`, column
// shift dx, K step s (16 channels).
template <int CI>
__host__ __device__ constexpr uint32_t conv_a_off(int slot, int dx, int s) {
    return (uint32_t)(((slot * (CI / 8) + 2 * s) * TC_APAD + dx) * 16);
}
// Offset of the B operand (weights) of tap t, K step s.
template <int CI, int CO>
__host__ __device__ constexpr uint32_t conv_b_off(int tap, int s) {
    return (uint32_t)((tap * (CI / 8) + 2 * s) * CO * 16);
}
template <int CO>
__host__ __device__ constexpr uint32_t conv_b_lbo() {
    return (uint32_t)CO * 16;
}

// Shared-memory matrix descriptor, no swizzling: 14-bit start address, the
// leading (K-direction, between 8 x 16-byte core matrices) and stride
// (M/N-direction, between 8-row groups) byte offsets, all in 16-byte units;
// bit 46 is the descriptor version of this MMA generation; base offset,
// offset mode and swizzle mode (bits 49-52, 61-63) are 0.
__host__ __device__ constexpr uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo & 0x3FFFFu) >> 4) << 16) |
           ((uint64_t)((sbo & 0x3FFFFu) >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor of a dense BF16 x BF16 -> FP32 MMA with both
// operands K-major: D format F32 (bits 4-5), A and B format BF16 (bits 7-9,
// 10-12), N / 8 (bits 17-22), M / 16 (bits 24-28).
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

}  // namespace swe
