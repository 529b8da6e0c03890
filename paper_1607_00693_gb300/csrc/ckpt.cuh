// Byte-buffer checkpoints of the library's handles: an 8-byte magic tag, a
// format version and an endianness probe, then fixed-width fields and arrays
// in a fixed order.  Host code only.
#pragma once
#include <stdint.h>
#include <stddef.h>
#include <string.h>

namespace stomsfem {

constexpr uint32_t kCkptVersion = 1;
constexpr uint32_t kCkptEndian = 0x01020304u;

// Writes into buf (when it is non-NULL and large enough) and counts bytes.
struct CkptWriter {
  unsigned char* buf;
  size_t cap, pos = 0;
  CkptWriter(void* b, size_t c) : buf(static_cast<unsigned char*>(b)), cap(c) {}
  bool fits() const { return buf && pos <= cap; }
  void put(const void* src, size_t n) {
    if (buf && pos + n <= cap) memcpy(buf + pos, src, n);
    pos += n;
  }
  template <typename T>
  void val(const T& v) { put(&v, sizeof(T)); }
  // host-side staging of a device array is done by the caller: `put` of host data
};

struct CkptReader {
  const unsigned char* buf;
  size_t cap, pos = 0;
  bool ok = true;
  CkptReader(const void* b, size_t c) : buf(static_cast<const unsigned char*>(b)), cap(c) {}
  void get(void* dst, size_t n) {
    if (!ok || pos + n > cap) {
      ok = false;
      return;
    }
    memcpy(dst, buf + pos, n);
    pos += n;
  }
  template <typename T>
  T val() {
    T v{};
    get(&v, sizeof(T));
    return v;
  }
};

inline void ckpt_header(CkptWriter& w, const char magic[8]) {
  w.put(magic, 8);
  w.val<uint32_t>(kCkptVersion);
  w.val<uint32_t>(kCkptEndian);
}

// 0: header matches; 1: not this kind of checkpoint or another version/byte order; 2: truncated.
inline int ckpt_check_header(CkptReader& r, const char magic[8]) {
  char m[8];
  r.get(m, 8);
  const uint32_t ver = r.val<uint32_t>(), end = r.val<uint32_t>();
  if (!r.ok) return 2;
  if (memcmp(m, magic, 8) != 0 || ver != kCkptVersion || end != kCkptEndian) return 1;
  return 0;
}

}  // namespace stomsfem
