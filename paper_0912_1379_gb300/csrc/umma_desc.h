// Encoders of the two descriptors a tcgen05.mma instruction takes (the PTX
// ISA's "shared memory descriptor" and "instruction descriptor" for the
// 5th-generation tensor cores), as plain constexpr C++ so that the host
// tests can check every field without a GPU.
//
// Shared-memory matrix descriptor (64 bits), K-major operand without
// swizzling.  The operand is stored as "core matrices" of 8 rows x 16 bytes
// (8 rows of 4 TF32 / 8 BF16 values), each core matrix 128 contiguous bytes
// (row r at byte 16 r).  Core matrices adjacent along K are LBO bytes apart,
// core matrices adjacent along M (or N) -- the next 8 rows -- SBO bytes apart.
//   bits  0-13  start address >> 4
//   bits 16-29  leading-dimension byte offset (LBO) >> 4
//   bits 32-45  stride-dimension byte offset (SBO) >> 4
//   bits 46-47  descriptor version, 1
//   bits 49-51  base offset (0: no swizzle pattern to align)
//   bit  52     LBO mode (0)
//   bits 61-63  layout: 0 = no swizzle
//
// Instruction descriptor (32 bits) of kind::tf32 / kind::f16:
//   bits  4-5   accumulator format (1 = F32)
//   bits  7-9   A format, bits 10-12 B format (kind::f16: 0 = F16, 1 = BF16;
//               kind::tf32: 2 = TF32)
//   bit  13/14  negate A / B (0)
//   bit  15/16  A / B major (0 = K-major)
//   bits 17-22  N >> 3
//   bits 24-28  M >> 4
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define UMMA_HD __host__ __device__
#else
#define UMMA_HD
#endif

namespace umma {

constexpr uint32_t kFmtF16 = 0, kFmtBF16 = 1, kFmtTF32 = 2, kAccF32 = 1;

UMMA_HD constexpr uint64_t smem_desc(uint32_t start_addr, uint32_t lbo_bytes, uint32_t sbo_bytes) {
    return (uint64_t)((start_addr >> 4) & 0x3FFFu) |
           ((uint64_t)((lbo_bytes >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo_bytes >> 4) & 0x3FFFu) << 32) |
           ((uint64_t)1 << 46);
}

UMMA_HD constexpr uint32_t instr_desc(uint32_t a_fmt, uint32_t b_fmt, uint32_t m, uint32_t n) {
    return (kAccF32 << 4) | (a_fmt << 7) | (b_fmt << 10) | ((n >> 3) << 17) | ((m >> 4) << 24);
}

// Byte offset of element (r, k) of a K-major operand tile laid out as above,
// with 4-byte elements (TF32), core matrices of 4 K values, LBO = 128 bytes
// (the core matrices of one 8-row group contiguous along K) and SBO = the
// bytes of one 8-row group (128 x K / 4).
UMMA_HD constexpr uint32_t tf32_offset(uint32_t r, uint32_t k, uint32_t k_tile) {
    return (r >> 3) * (k_tile * 32u) + (k >> 2) * 128u + (r & 7u) * 16u + (k & 3u) * 4u;
}

}  // namespace umma
