// Index checkpoint files: a fixed header followed by the index's device arrays,
// streamed through one page-locked host buffer.  Host code only.
//
// File layout (native byte order):
//   CkptHeader
//   array 0 bytes, array 1 bytes, ...     (as listed by the writer)
// The header's checksum is a 64-bit multiply-xor hash over the arrays' 8-byte
// words, in file order (the arrays are multiples of 8 bytes long).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <cstring>

#include "slash.h"

namespace slash {

constexpr char kCkptMagic[8] = {'S', 'L', 'A', 'S', 'H', 'I', 'X', '1'};
constexpr uint32_t kCkptReservoir = 0u;  // slash_index: fill [nk] then slots [nk][R]
constexpr uint32_t kCkptSketch = 1u;     // slash_tk_index: cells [nk][W][C]

struct CkptHeader {
  char magic[8];
  uint32_t kind;
  uint32_t header_bytes;   // sizeof(CkptHeader), for a later format to grow
  uint32_t params[16];     // the kind's parameter struct, as raw words (zero-padded)
  uint64_t next_id;
  uint64_t payload_bytes;  // sum of the arrays' sizes
  uint64_t checksum;
};

struct DevSpan {
  void* ptr;
  uint64_t bytes;
};

inline uint64_t ckpt_hash(uint64_t h, const void* data, size_t bytes) {
  const unsigned char* p = static_cast<const unsigned char*>(data);
  for (size_t i = 0; i + 8 <= bytes; i += 8) {
    uint64_t w;
    std::memcpy(&w, p + i, 8);
    h = (h ^ w) * 0x100000001B3ull;
    h ^= h >> 29;
  }
  return h;
}

constexpr uint64_t kCkptChunk = 64ull << 20;  // staging buffer size

// Writes the header and the arrays; synchronises the device.  Returns SLASH_OK,
// SLASH_EIO (file) or SLASH_ECUDA / SLASH_ENOMEM (copies, staging buffer).
inline int ckpt_save(const char* path, CkptHeader hdr, const DevSpan* spans, int n) {
  if (cudaDeviceSynchronize() != cudaSuccess) return SLASH_ECUDA;
  void* buf = nullptr;
  if (cudaMallocHost(&buf, kCkptChunk) != cudaSuccess) { cudaGetLastError(); return SLASH_ENOMEM; }
  FILE* f = std::fopen(path, "wb");
  int rc = f ? SLASH_OK : SLASH_EIO;
  std::memcpy(hdr.magic, kCkptMagic, 8);
  hdr.header_bytes = sizeof(CkptHeader);
  hdr.payload_bytes = 0;
  hdr.checksum = 0xCBF29CE484222325ull;
  for (int i = 0; i < n; ++i) hdr.payload_bytes += spans[i].bytes;
  // header first (checksum patched at the end)
  if (rc == SLASH_OK && std::fwrite(&hdr, sizeof hdr, 1, f) != 1) rc = SLASH_EIO;
  for (int i = 0; i < n && rc == SLASH_OK; ++i) {
    for (uint64_t off = 0; off < spans[i].bytes && rc == SLASH_OK; off += kCkptChunk) {
      const uint64_t b = spans[i].bytes - off < kCkptChunk ? spans[i].bytes - off : kCkptChunk;
      if (cudaMemcpy(buf, static_cast<char*>(spans[i].ptr) + off, b, cudaMemcpyDeviceToHost) != cudaSuccess) {
        rc = SLASH_ECUDA;
        break;
      }
      hdr.checksum = ckpt_hash(hdr.checksum, buf, b);
      if (std::fwrite(buf, 1, b, f) != b) rc = SLASH_EIO;
    }
  }
  if (rc == SLASH_OK && (std::fseek(f, 0, SEEK_SET) != 0 || std::fwrite(&hdr, sizeof hdr, 1, f) != 1))
    rc = SLASH_EIO;
  if (f && std::fclose(f) != 0 && rc == SLASH_OK) rc = SLASH_EIO;
  cudaFreeHost(buf);
  return rc;
}

// Reads and checks the header (magic, kind, sizes).  Leaves *f positioned at the
// first array.  Returns SLASH_OK, SLASH_EIO (cannot open / short read) or
// SLASH_EINVAL (not a checkpoint of this kind).
inline int ckpt_open(const char* path, uint32_t kind, CkptHeader* hdr, FILE** f) {
  *f = std::fopen(path, "rb");
  if (!*f) return SLASH_EIO;
  if (std::fread(hdr, sizeof *hdr, 1, *f) != 1) { std::fclose(*f); *f = nullptr; return SLASH_EINVAL; }
  if (std::memcmp(hdr->magic, kCkptMagic, 8) != 0 || hdr->kind != kind || hdr->header_bytes != sizeof *hdr) {
    std::fclose(*f);
    *f = nullptr;
    return SLASH_EINVAL;
  }
  return SLASH_OK;
}

// Streams the arrays into device memory and checks the checksum; closes f.
inline int ckpt_load(FILE* f, const CkptHeader& hdr, const DevSpan* spans, int n) {
  uint64_t total = 0;
  for (int i = 0; i < n; ++i) total += spans[i].bytes;
  if (total != hdr.payload_bytes) { std::fclose(f); return SLASH_EINVAL; }
  void* buf = nullptr;
  if (cudaMallocHost(&buf, kCkptChunk) != cudaSuccess) { cudaGetLastError(); std::fclose(f); return SLASH_ENOMEM; }
  uint64_t h = 0xCBF29CE484222325ull;
  int rc = SLASH_OK;
  for (int i = 0; i < n && rc == SLASH_OK; ++i) {
    for (uint64_t off = 0; off < spans[i].bytes && rc == SLASH_OK; off += kCkptChunk) {
      const uint64_t b = spans[i].bytes - off < kCkptChunk ? spans[i].bytes - off : kCkptChunk;
      if (std::fread(buf, 1, b, f) != b) { rc = SLASH_EINVAL; break; }  // truncated
      h = ckpt_hash(h, buf, b);
      if (cudaMemcpy(static_cast<char*>(spans[i].ptr) + off, buf, b, cudaMemcpyHostToDevice) != cudaSuccess)
        rc = SLASH_ECUDA;
    }
  }
  if (rc == SLASH_OK && h != hdr.checksum) rc = SLASH_EINVAL;
  if (rc == SLASH_OK && std::fgetc(f) != EOF) rc = SLASH_EINVAL;  // trailing bytes
  std::fclose(f);
  cudaFreeHost(buf);
  return rc;
}

}  // namespace slash
