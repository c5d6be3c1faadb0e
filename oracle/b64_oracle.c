/*
 * Scalar CPU oracle for base64 encoding and decoding (Muła & Lemire,
 * "Faster Base64 Encoding and Decoding using AVX2 Instructions").
 *
 * TEST INFRASTRUCTURE ONLY. This file is the checker that the CUDA codec is
 * compared against. Only the tests, the smoke check and the benchmark's CPU
 * baseline load it; the product library never links or calls it, and it
 * shares no code, table or header with the CUDA sources.
 *
 * It is deliberately plain: one byte or character at a time, integer
 * division and modulo exactly as the paper writes them, no tables other than
 * the paper's Table 1, no blocking and no vectorisation.
 *
 *   oracle_encode  - Algorithm 1 (Section 2), with B given by Table 1.
 *   oracle_decode  - Algorithm 2 (Section 2), with A the inverse of Table 1,
 *                    made strict as Section 2 asks ("report an error when
 *                    characters outside of this set are encountered") and
 *                    as Appendix B restates from RFC 4648.
 *
 * Readings where the paper is silent or inconsistent (each one is listed in
 * the design notes of this repository):
 *   R1  '=' is accepted only as the last character, or as the last two
 *       characters, of an input whose length is a multiple of 4. Any other
 *       '=' is an invalid character (Algorithm 2 would give it value 0).
 *   R2  A length that is not a multiple of 4 (Algorithm 2 only requires it)
 *       gives status BAD_LENGTH and first_bad = m - (m mod 4), the start of
 *       the incomplete group, unless an invalid character comes first; the
 *       invalid-character scan covers the whole input and wins.
 *   R3  Non-zero trailing bits in the last group (Appendix A) are accepted
 *       and dropped; the paper notes the standard does not require the check.
 *   R4  Whitespace is not removed (Section 2.3 says it must be removed before
 *       decoding); it is an invalid character here.
 *
 * Parity pins (tests/test_oracle_pins.py): Python's base64/binascii on all
 * 2^24 three-byte groups and all 64^4 valid quads, the paper's worked
 * examples (Section 2.2, Section 2.3, Appendix C), Appendix C's nibble
 * bitsets against Table 1 over all 256 bytes, strict-mode accept/reject
 * against binascii, and first_bad by construction on injected errors.
 */
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>

/* Status codes of the decoder (same numbering as the C ABI, written out
 * separately here so that the oracle depends on nothing of the product). */
#define ORACLE_OK 0
#define ORACLE_INVALID_CHAR 1
#define ORACLE_BAD_LENGTH 2

/* Table 1: the 6-bit value v is represented by the character TABLE1[v]. */
static const char TABLE1[64] = {
    'A', 'B', 'C', 'D', 'E', 'F', 'G', 'H', 'I', 'J', 'K', 'L', 'M',
    'N', 'O', 'P', 'Q', 'R', 'S', 'T', 'U', 'V', 'W', 'X', 'Y', 'Z',
    'a', 'b', 'c', 'd', 'e', 'f', 'g', 'h', 'i', 'j', 'k', 'l', 'm',
    'n', 'o', 'p', 'q', 'r', 's', 't', 'u', 'v', 'w', 'x', 'y', 'z',
    '0', '1', '2', '3', '4', '5', '6', '7', '8', '9', '+', '/'};

#define PAD '='

/* B of Algorithm 1: value in [0,64) -> character (Table 1). */
static char B(unsigned v) { return TABLE1[v]; }

/* A of Algorithm 2: character -> value in [0,64), or -1 when the character is
 * not in Table 1. Linear search over Table 1, so it is Table 1 by definition. */
static int A(unsigned char x) {
  for (int v = 0; v < 64; v++)
    if ((unsigned char)TABLE1[v] == x) return v;
  return -1;
}

int oracle_table1_value(unsigned char x) { return A(x); }
char oracle_table1_char(unsigned v) { return v < 64 ? B(v) : 0; }

/* Output length of Algorithm 1: four characters per started group of three
 * bytes (Section 2). */
size_t oracle_encoded_len(size_t n) { return 4 * (n / 3 + (n % 3 != 0)); }

/* Algorithm 1. Writes oracle_encoded_len(n) characters to p (no terminator)
 * and returns that count. */
size_t oracle_encode(const uint8_t *s, size_t n, char *p) {
  size_t k = 0;
  size_t i;
  /* main loop over i = 0, 3, ..., n - (n mod 3) - 3 */
  for (i = 0; i + 3 <= n - (n % 3); i += 3) {
    p[k++] = B(s[i] / 4);
    p[k++] = B(((s[i] * 16) % 64) + (s[i + 1] / 16));
    p[k++] = B(((s[i + 1] * 4) % 64) + (s[i + 2] / 64));
    p[k++] = B(s[i + 2] % 64);
  }
  i = n - n % 3;
  if (i < n) {
    p[k++] = B(s[i] / 4);
    if (i == n - 1) {
      p[k++] = B((s[i] * 16) % 64);
      p[k++] = PAD;
    } else if (i == n - 2) {
      p[k++] = B(((s[i] * 16) % 64) + (s[i + 1] / 16));
      p[k++] = B((s[i + 1] * 4) % 64);
    }
    p[k++] = PAD;
  }
  return k;
}

/* Capacity a decode of m characters may write: three bytes per complete
 * group of four characters. */
size_t oracle_decoded_cap(size_t m) { return 3 * (m / 4); }

/* Number of trailing characters that R1 accepts as padding. */
static size_t padding_count(const char *c, size_t m) {
  if (m < 4 || m % 4 != 0) return 0;
  if (c[m - 1] != PAD) return 0;
  if (c[m - 2] != PAD) return 1;
  return 2;
}

/* Algorithm 2 with readings R1-R4. On success writes 3*(m/4) - |P| bytes,
 * sets *first_bad = m and returns ORACLE_OK. On failure writes nothing
 * useful, sets *outlen = 0 and *first_bad as in R1/R2. */
int oracle_decode(const char *c, size_t m, uint8_t *p, size_t *outlen,
                  size_t *first_bad) {
  size_t npad = padding_count(c, m);
  /* invalid characters: outside Table 1 and not an accepted padding '=' */
  for (size_t i = 0; i < m; i++) {
    int is_padding = (npad > 0) && (i >= m - npad);
    if (A((unsigned char)c[i]) < 0 && !is_padding) {
      *first_bad = i;
      *outlen = 0;
      return ORACLE_INVALID_CHAR;
    }
  }
  if (m % 4 != 0) {
    *first_bad = m - m % 4;
    *outlen = 0;
    return ORACLE_BAD_LENGTH;
  }
  size_t k = 0;
  for (size_t i = 0; i + 4 <= m; i += 4) {
    /* the padding character has value 0 (Algorithm 2's convention) */
    int a = A((unsigned char)c[i]);
    int b = A((unsigned char)c[i + 1]);
    int cc = (c[i + 2] == PAD) ? 0 : A((unsigned char)c[i + 2]);
    int d = (c[i + 3] == PAD) ? 0 : A((unsigned char)c[i + 3]);
    p[k++] = (uint8_t)((a * 4) + (b / 16));
    if (c[i + 2] == PAD) break;
    p[k++] = (uint8_t)(((b * 16) % 256) + (cc / 4));
    if (c[i + 3] == PAD) break;
    p[k++] = (uint8_t)(((cc * 64) % 256) + d);
  }
  *outlen = k;
  *first_bad = m;
  return ORACLE_OK;
}

/* Many messages packed back to back; in_off[0..nmsg] are exclusive prefix
 * offsets into src. Output j starts at out_off[j], the prefix of
 * oracle_encoded_len over the messages before it. */
void oracle_encode_batch(const uint8_t *src, const int64_t *in_off,
                         int64_t nmsg, char *dst, int64_t *out_off) {
  out_off[0] = 0;
  for (int64_t j = 0; j < nmsg; j++) {
    size_t n = (size_t)(in_off[j + 1] - in_off[j]);
    out_off[j + 1] = out_off[j] + (int64_t)oracle_encoded_len(n);
    oracle_encode(src + in_off[j], n, dst + out_off[j]);
  }
}

/* Decode of many packed messages. Output j starts at out_off[j], the prefix
 * of oracle_decoded_cap; status, first_bad (relative to the message start)
 * and outlen are per message. */
void oracle_decode_batch(const char *src, const int64_t *in_off, int64_t nmsg,
                         uint8_t *dst, int64_t *out_off, int32_t *status,
                         int64_t *first_bad, int64_t *outlen) {
  out_off[0] = 0;
  for (int64_t j = 0; j < nmsg; j++) {
    size_t m = (size_t)(in_off[j + 1] - in_off[j]);
    size_t ol = 0, fb = 0;
    out_off[j + 1] = out_off[j] + (int64_t)oracle_decoded_cap(m);
    status[j] = oracle_decode(src + in_off[j], m, dst + out_off[j], &ol, &fb);
    first_bad[j] = (int64_t)fb;
    outlen[j] = (int64_t)ol;
  }
}

/* ------------------------------------------------------------------------
 * Variants (Section 2 and Appendix A), selected by flags:
 *   ORACLE_FLAG_URL          base64url: value 62 is '-' and value 63 is '_'
 *                            instead of '+' and '/' (Section 2).
 *   ORACLE_FLAG_NOPAD        padding omitted (Section 2: acceptable when the
 *                            size of the data is otherwise known): encode
 *                            writes no '='; decode also accepts a final group
 *                            of 2 or 3 characters (1 or 2 bytes). A final
 *                            group of 1 character is still BAD_LENGTH.
 *   ORACLE_FLAG_STRICT_TAIL  Appendix A: with two padding characters (or a
 *                            2-character final group) (A(c) * 16) mod 256 = 0
 *                            for the last data character c; with one (or a
 *                            3-character final group) (A(c) * 64) mod 256 =
 *                            0. A violation is status NONCANONICAL with
 *                            first_bad = the index of c.
 * With flags = 0 these functions compute exactly oracle_encode and
 * oracle_decode (checked by the tests).
 * ---------------------------------------------------------------------- */
#define ORACLE_FLAG_URL 1
#define ORACLE_FLAG_NOPAD 2
#define ORACLE_FLAG_STRICT_TAIL 4
#define ORACLE_NONCANONICAL 3

/* B and A of the selected alphabet. */
static char B_ex(unsigned v, int flags) {
  if (flags & ORACLE_FLAG_URL) {
    if (v == 62) return '-';
    if (v == 63) return '_';
  }
  return B(v);
}

static int A_ex(unsigned char x, int flags) {
  if (flags & ORACLE_FLAG_URL) {
    if (x == '-') return 62;
    if (x == '_') return 63;
    if (x == '+' || x == '/') return -1;
  }
  return A(x);
}

size_t oracle_encoded_len_ex(size_t n, int flags) {
  if (flags & ORACLE_FLAG_NOPAD) return 4 * (n / 3) + (n % 3 ? n % 3 + 1 : 0);
  return oracle_encoded_len(n);
}

/* Algorithm 1 with the alphabet of `flags`; under NOPAD the padding
 * characters are not appended. */
size_t oracle_encode_ex(const uint8_t *s, size_t n, char *p, int flags) {
  const int pad = !(flags & ORACLE_FLAG_NOPAD);
  size_t k = 0;
  size_t i;
  for (i = 0; i + 3 <= n - (n % 3); i += 3) {
    p[k++] = B_ex(s[i] / 4, flags);
    p[k++] = B_ex(((s[i] * 16) % 64) + (s[i + 1] / 16), flags);
    p[k++] = B_ex(((s[i + 1] * 4) % 64) + (s[i + 2] / 64), flags);
    p[k++] = B_ex(s[i + 2] % 64, flags);
  }
  i = n - n % 3;
  if (i < n) {
    p[k++] = B_ex(s[i] / 4, flags);
    if (i == n - 1) {
      p[k++] = B_ex((s[i] * 16) % 64, flags);
      if (pad) p[k++] = PAD;
    } else if (i == n - 2) {
      p[k++] = B_ex(((s[i] * 16) % 64) + (s[i + 1] / 16), flags);
      p[k++] = B_ex((s[i + 1] * 4) % 64, flags);
    }
    if (pad) p[k++] = PAD;
  }
  return k;
}

size_t oracle_decoded_cap_ex(size_t m, int flags) {
  size_t cap = 3 * (m / 4);
  if ((flags & ORACLE_FLAG_NOPAD) && m % 4 >= 2) cap += m % 4 - 1;
  return cap;
}

/* Algorithm 2 with readings R1-R4, the alphabet of `flags`, optional
 * padding (NOPAD) and Appendix A's check (STRICT_TAIL). */
int oracle_decode_ex(const char *c, size_t m, uint8_t *p, size_t *outlen, size_t *first_bad,
                     int flags) {
  const int nopad = (flags & ORACLE_FLAG_NOPAD) != 0;
  size_t npad = padding_count(c, m);
  for (size_t i = 0; i < m; i++) {
    int is_padding = (npad > 0) && (i >= m - npad);
    if (A_ex((unsigned char)c[i], flags) < 0 && !is_padding) {
      *first_bad = i;
      *outlen = 0;
      return ORACLE_INVALID_CHAR;
    }
  }
  if (m % 4 != 0 && (!nopad || m % 4 == 1)) {
    *first_bad = m - m % 4;
    *outlen = 0;
    return ORACLE_BAD_LENGTH;
  }
  /* Appendix A on the last data character (padded or unpadded tail) */
  if (flags & ORACLE_FLAG_STRICT_TAIL) {
    size_t rest = nopad ? m % 4 : 0; /* characters of an unpadded final group */
    size_t idx = 0;
    int mult = 0;
    if (npad == 2 || rest == 2) {
      idx = (npad == 2) ? m - 3 : m - 1;
      mult = 16;
    } else if (npad == 1 || rest == 3) {
      idx = (npad == 1) ? m - 2 : m - 1;
      mult = 64;
    }
    if (mult && (A_ex((unsigned char)c[idx], flags) * mult) % 256 != 0) {
      *first_bad = idx;
      *outlen = 0;
      return ORACLE_NONCANONICAL;
    }
  }
  size_t k = 0;
  const size_t whole = m - m % 4;
  for (size_t i = 0; i + 4 <= whole; i += 4) {
    int a = A_ex((unsigned char)c[i], flags);
    int b = A_ex((unsigned char)c[i + 1], flags);
    int cc = (c[i + 2] == PAD) ? 0 : A_ex((unsigned char)c[i + 2], flags);
    int d = (c[i + 3] == PAD) ? 0 : A_ex((unsigned char)c[i + 3], flags);
    p[k++] = (uint8_t)((a * 4) + (b / 16));
    if (c[i + 2] == PAD) break;
    p[k++] = (uint8_t)(((b * 16) % 256) + (cc / 4));
    if (c[i + 3] == PAD) break;
    p[k++] = (uint8_t)(((cc * 64) % 256) + d);
  }
  if (m % 4 >= 2) { /* unpadded final group (NOPAD) */
    int a = A_ex((unsigned char)c[whole], flags);
    int b = A_ex((unsigned char)c[whole + 1], flags);
    p[k++] = (uint8_t)((a * 4) + (b / 16));
    if (m % 4 == 3) {
      int cc = A_ex((unsigned char)c[whole + 2], flags);
      p[k++] = (uint8_t)(((b * 16) % 256) + (cc / 4));
    }
  }
  *outlen = k;
  *first_bad = m;
  return ORACLE_OK;
}

/* ------------------------------------------------------------------------
 * Whitespace (Appendix B): with ORACLE_FLAG_SKIP_WS the decoder first
 * removes the space, line-feed and carriage-return characters, the way
 * Fig. 11 does (copy every byte, advance the write position only for bytes
 * that are kept), remembering where each kept byte came from; it decodes
 * the remaining characters with the other flags and reports first_bad as
 * an index into the original input (m, the original length, on success).
 * ---------------------------------------------------------------------- */
#define ORACLE_FLAG_SKIP_WS 8

static int is_space(unsigned char x) { return x == ' ' || x == '\n' || x == '\r'; }

int oracle_decode_ws(const char *c, size_t m, uint8_t *p, size_t *outlen, size_t *first_bad,
                     int flags) {
  char *kept = (char *)malloc(m ? m : 1);
  size_t *from = (size_t *)malloc((m ? m : 1) * sizeof(size_t));
  if (!kept || !from) {
    free(kept);
    free(from);
    return -3;
  }
  size_t q = 0;
  for (size_t i = 0; i < m; i++) {
    kept[q] = c[i];
    from[q] = i;
    q += !is_space((unsigned char)c[i]);
  }
  size_t fb = 0;
  int st = oracle_decode_ex(kept, q, p, outlen, &fb, flags & ~ORACLE_FLAG_SKIP_WS);
  *first_bad = (st == ORACLE_OK) ? m : from[fb];
  free(kept);
  free(from);
  return st;
}
