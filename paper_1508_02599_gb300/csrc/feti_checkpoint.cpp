// Checkpoints of load-stepped runs: the state (U, load step, tau) after a
// completed load step of the Newton method of Sec. 3.2 (Eq. loadStepping), so
// that a long run -- hundreds of load steps, as in the study of Sec. 5.3 -- can
// stop and resume with feti_newton_steps from the next step.
//
// File layout (native byte order; little-endian on the supported hosts):
//   8 bytes  magic "FETICKP1"
//   int64    n_dofs
//   int32    step (the last completed load step)
//   int32    n_load_steps
//   double   tau = step / n_load_steps
//   double   U[n_dofs]
//   uint64   FNV-1a hash of every byte before it
// Written to "<path>.tmp" and renamed over path, so a reader sees either the
// previous complete file or the new one.  Host code only: no CUDA call.
#include "feti.h"

#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

namespace {

constexpr char kMagic[8] = {'F', 'E', 'T', 'I', 'C', 'K', 'P', '1'};

struct Fnv {
  uint64_t h = 1469598103934665603ull;
  void add(const void* p, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) {
      h ^= b[i];
      h *= 1099511628211ull;
    }
  }
};

struct File {
  FILE* f = nullptr;
  ~File() {
    if (f) std::fclose(f);
  }
};

}  // namespace

extern "C" {

feti_status feti_checkpoint_write(const char* path, const double* U, int64_t n_dofs, int32_t step,
                                  int32_t n_load_steps, double tau) {
  if (!path || !U || n_dofs <= 0 || step < 0 || n_load_steps <= 0 || step > n_load_steps)
    return FETI_ERR_INVALID_ARG;
  const std::string tmp = std::string(path) + ".tmp";
  Fnv h;
  {
    File out;
    out.f = std::fopen(tmp.c_str(), "wb");
    if (!out.f) return FETI_ERR_IO;
    auto put = [&](const void* p, size_t n) {
      h.add(p, n);
      return std::fwrite(p, 1, n, out.f) == n;
    };
    bool ok = put(kMagic, sizeof(kMagic)) && put(&n_dofs, sizeof(n_dofs)) && put(&step, sizeof(step)) &&
              put(&n_load_steps, sizeof(n_load_steps)) && put(&tau, sizeof(tau)) &&
              put(U, sizeof(double) * (size_t)n_dofs);
    const uint64_t digest = h.h;
    ok = ok && std::fwrite(&digest, 1, sizeof(digest), out.f) == sizeof(digest);
    ok = ok && std::fflush(out.f) == 0;
    if (std::fclose(out.f) != 0) ok = false;
    out.f = nullptr;
    if (!ok) {
      std::remove(tmp.c_str());
      return FETI_ERR_IO;
    }
  }
  if (std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    return FETI_ERR_IO;
  }
  return FETI_OK;
}

feti_status feti_checkpoint_read(const char* path, double* U, int64_t capacity, feti_checkpoint_info* info) {
  if (!path) return FETI_ERR_INVALID_ARG;
  File in;
  in.f = std::fopen(path, "rb");
  if (!in.f) return FETI_ERR_IO;
  Fnv h;
  auto get = [&](void* p, size_t n) {
    if (std::fread(p, 1, n, in.f) != n) return false;
    h.add(p, n);
    return true;
  };
  char magic[8];
  feti_checkpoint_info ci{};
  if (!get(magic, sizeof(magic)) || std::memcmp(magic, kMagic, sizeof(kMagic)) != 0) return FETI_ERR_IO;
  if (!get(&ci.n_dofs, sizeof(ci.n_dofs)) || !get(&ci.step, sizeof(ci.step)) ||
      !get(&ci.n_load_steps, sizeof(ci.n_load_steps)) || !get(&ci.tau, sizeof(ci.tau)))
    return FETI_ERR_IO;
  if (ci.n_dofs <= 0 || ci.n_load_steps <= 0 || ci.step < 0 || ci.step > ci.n_load_steps) return FETI_ERR_IO;
  if (info) *info = ci;
  if (!U) return FETI_OK;  // header only
  if (capacity < ci.n_dofs) return FETI_ERR_INVALID_ARG;
  std::vector<double> buf((size_t)ci.n_dofs);
  if (!get(buf.data(), sizeof(double) * buf.size())) return FETI_ERR_IO;
  uint64_t digest = 0;
  if (std::fread(&digest, 1, sizeof(digest), in.f) != sizeof(digest) || digest != h.h) return FETI_ERR_IO;
  std::memcpy(U, buf.data(), sizeof(double) * buf.size());
  return FETI_OK;
}

}  // extern "C"
