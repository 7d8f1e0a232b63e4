// Index checks of the debug build.  Compiled with -DFX_BOUNDS_CHECK, FXI(i, n) checks an index i
// into a buffer of n elements.  An index outside [0, n) sets ST_BOUNDS in the launch's status word
// (A.status: every kernel that uses these marks names its launch arguments A); the first such
// index of the run records its site (a 16-bit tag of the source file's name, then the line), the
// index and n in the words that follow the status bits; and the access goes to element 0 of the
// buffer instead, which keeps it inside the buffer.  Nothing traps or waits.
//   FXI_AT(st, i, n)      as FXI, with the status word st (code outside a kernel's body);
//   FXP(p, off, n)        the address p + off, off checked as FXI checks an index (FXP_AT: with st);
//   FXPR(p, off, len, n)  the start of the range [off, off + len) that a helper walks (len <= n; a
//                         range that does not fit starts at p).
// In the normal build each is its plain index or address and costs nothing.
//
// Layout of the status region (unsigned words, 8-byte aligned): [0] status bits, [1] site of the
// first out-of-range index, [2..3] that index (int64), [4..5] the buffer's extent (int64).
#pragma once
#include <stdint.h>

#include <type_traits>

#include "fx_types.h"

namespace fx {

// FNV-1a hash of a path's base name folded to 16 bits; the host maps it back to a file name.
__host__ __device__ constexpr unsigned fxb_file_tag(const char* path) {
  const char* b = path;
  for (const char* p = path; *p; ++p)
    if (*p == '/') b = p + 1;
  unsigned h = 2166136261u;
  for (const char* p = b; *p; ++p) {
    h ^= (unsigned char)*p;
    h *= 16777619u;
  }
  return (h ^ (h >> 16)) & 0xffffu;
}

#ifdef FX_BOUNDS_CHECK
static __device__ __noinline__ void fxb_record(unsigned* st, unsigned site, long long i, long long n) {
  if (atomicCAS(st + 1, 0u, site) == 0u) {
    reinterpret_cast<long long*>(st)[1] = i;
    reinterpret_cast<long long*>(st)[2] = n;
  }
  atomicOr(st, ST_BOUNDS);
}
template <class I>
__device__ __forceinline__ I fxb_index(unsigned* st, unsigned site, I i, long long n) {
  if ((unsigned long long)(long long)i < (unsigned long long)n) return i;
  fxb_record(st, site, (long long)i, n);
  return I(0);
}
template <class I>
__device__ __forceinline__ I fxb_range(unsigned* st, unsigned site, I off, long long len, long long n) {
  if ((long long)off >= 0 && (long long)off + len <= n) return off;
  fxb_record(st, site, (long long)off + len - 1, n);
  return I(0);
}
#define FXB_SITE ((std::integral_constant<unsigned, ::fx::fxb_file_tag(__FILE__)>::value << 16) | (unsigned)__LINE__)
#define FXI_AT(st, i, n) ::fx::fxb_index((st), FXB_SITE, (i), (long long)(n))
#define FXP_AT(st, p, off, n) ((p) + ::fx::fxb_index((st), FXB_SITE, (off), (long long)(n)))
#define FXPR(p, off, len, n) ((p) + ::fx::fxb_range(A.status, FXB_SITE, (off), (long long)(len), (long long)(n)))
#else
// (p + off without parentheses: the same tokens, and so the same code, as the unchecked source)
#define FXI_AT(st, i, n) (i)
#define FXP_AT(st, p, off, n) p + off
#define FXPR(p, off, len, n) p + off
#endif
#define FXP(p, off, n) FXP_AT(A.status, p, off, n)
#define FXI(i, n) FXI_AT(A.status, i, n)

}  // namespace fx
