// Carving of caller-provided workspaces into 256-byte aligned arrays.
#pragma once

#include <stddef.h>
#include <stdint.h>

namespace aeqc {

constexpr size_t kWsAlign = 256;

inline size_t ws_round(size_t b) { return (b + kWsAlign - 1) / kWsAlign * kWsAlign; }

struct WsSize {
  size_t bytes = 0;
  template <typename T>
  void add(size_t count) {
    bytes += ws_round(count * sizeof(T));
  }
};

struct WsCarver {
  char* p;
  size_t left;
  bool good = true;
  WsCarver(char* base, size_t bytes) : p(base), left(bytes) {
    if (reinterpret_cast<uintptr_t>(base) % kWsAlign) good = false;
  }
  template <typename T>
  T* take(size_t count) {
    size_t b = ws_round(count * sizeof(T));
    if (!good || b > left) {
      good = false;
      return nullptr;
    }
    T* r = reinterpret_cast<T*>(p);
    p += b;
    left -= b;
    return r;
  }
  bool ok() const { return good; }
};

}  // namespace aeqc
