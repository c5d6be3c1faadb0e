// Length and status rules of the codec, shared by host and device code.
#pragma once

#include <cstdint>

#include "../../include/gb64.h"

#ifdef __CUDACC__
#define GB64_HD __host__ __device__
#else
#define GB64_HD
#endif

namespace gb64 {

// Codec variants (Section 2): base64url alphabet, omitted padding; and
// Appendix A's check of the final group.
constexpr uint32_t kFlagUrl = 1;
constexpr uint32_t kFlagNoPad = 2;
constexpr uint32_t kFlagStrictTail = 4;

// Output length of an encode and capacity of a decode under the flags.
GB64_HD constexpr uint64_t encoded_len_flags(uint64_t n, uint32_t flags) {
  return (flags & kFlagNoPad) ? 4 * (n / 3) + (n % 3 ? n % 3 + 1 : 0) : 4 * ((n + 2) / 3);
}
GB64_HD constexpr uint64_t decoded_cap_flags(uint64_t m, uint32_t flags) {
  return 3 * (m / 4) + (((flags & kFlagNoPad) && m % 4 >= 2) ? m % 4 - 1 : 0);
}

// Start of the final characters of a whole message of m characters.
GB64_HD inline uint64_t decode_body_end(uint64_t m) {
  if (m == 0) return 0;
  return (m % 4 == 0) ? m - 4 : m - m % 4;
}

// Status of a whole message once every character has been looked at
// (invalid character first, then the length rule, then Appendix A).
struct FinalStatus {
  int32_t status;
  int64_t first_bad;
  int64_t outlen;
};
GB64_HD inline FinalStatus final_status(uint64_t m, uint64_t body_end, unsigned long long min_bad,
                                        int64_t final, uint32_t flags) {
  const bool nopad_ok = (flags & kFlagNoPad) && m % 4 >= 2;
  if (min_bad != ~0ull && min_bad != 0x7FFFFFFFFFFFFFFFull)
    return FinalStatus{B64_ERR_INVALID_CHAR, (int64_t)min_bad, 0};
  if (m % 4 != 0 && !nopad_ok) return FinalStatus{B64_ERR_BAD_LENGTH, (int64_t)(m - m % 4), 0};
  if (final < 0)
    return FinalStatus{B64_ERR_NONCANONICAL, (int64_t)(body_end + (uint64_t)(-final - 1)), 0};
  return FinalStatus{B64_OK, (int64_t)m, (int64_t)(body_end / 4 * 3) + final};
}

}  // namespace gb64
