// MPS checkpoint files: mps_save / mps_load.
//
// File layout (little-endian, which both supported hosts are):
//   bytes 0..7     magic "VPMPS01\0"
//   bytes 8..11    int32 n (number of sites, 1..64)
//   bytes 12..15   int32 0 (reserved)
//   then           int32 ranks[n + 1], ranks[0] = ranks[n] = 1
//   then           zero padding to a multiple of 8 bytes
//   then           the cores as FP64, site after site, core k row-major
//                  (ranks[k], 2, ranks[k+1]) -- the packing of
//                  mps_get_cores / mps_create_cores.
// The bond ranks fix the payload size; a file whose size disagrees is
// rejected, so a truncated or padded file never loads.
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"

using vp::fail;

namespace {

const char kMagic[8] = {'V', 'P', 'M', 'P', 'S', '0', '1', '\0'};

struct File {
  FILE* f = nullptr;
  ~File() {
    if (f) fclose(f);
  }
};

size_t header_bytes(int n) {
  const size_t h = 16 + 4 * (size_t)(n + 1);
  return (h + 7) / 8 * 8;
}

size_t payload_elems(const std::vector<int>& r) {
  size_t e = 0;
  for (size_t k = 0; k + 1 < r.size(); ++k) e += (size_t)r[k] * 2 * r[k + 1];
  return e;
}

}  // namespace

extern "C" int mps_save(vp_ctx* ctx, const mps_t* m, const char* path) {
  if (!ctx || !m || !path) return fail(ctx, VP_EINVAL, "mps_save: bad argument");
  const int n = mps_num_sites(m);
  std::vector<int> r(n + 1);
  VP_TRY(mps_bonds(m, r.data()));
  std::vector<double> cores(payload_elems(r));
  VP_TRY(mps_get_cores(ctx, m, cores.data(), cores.size()));
  std::vector<char> head(header_bytes(n), 0);
  memcpy(head.data(), kMagic, 8);
  memcpy(head.data() + 8, &n, 4);
  memcpy(head.data() + 16, r.data(), 4 * (size_t)(n + 1));
  const std::string tmp = std::string(path) + ".tmp";
  {
    File fh;
    fh.f = fopen(tmp.c_str(), "wb");
    if (!fh.f) return fail(ctx, VP_EIO, std::string("mps_save: cannot open ") + tmp);
    if (fwrite(head.data(), 1, head.size(), fh.f) != head.size() ||
        fwrite(cores.data(), sizeof(double), cores.size(), fh.f) != cores.size() || fflush(fh.f) != 0)
      return fail(ctx, VP_EIO, std::string("mps_save: write failed on ") + tmp);
  }
  if (rename(tmp.c_str(), path) != 0) return fail(ctx, VP_EIO, std::string("mps_save: cannot rename to ") + path);
  return VP_OK;
}

// Header of a checkpoint file checked against the file's size before anything
// is allocated: a corrupt or hostile header that claims more payload than the
// file holds is rejected with VP_EIO.
static int bad(std::string& why, const char* what) {
  why = what;
  return VP_EIO;
}

static int read_header(FILE* f, int* n_out, std::vector<int>& r, size_t* elems_out, std::string& why) {
  char head[16];
  if (fread(head, 1, 16, f) != 16 || memcmp(head, kMagic, 8) != 0) return bad(why, "not an MPS file");
  int n = 0, reserved = 0;
  memcpy(&n, head + 8, 4);
  memcpy(&reserved, head + 12, 4);
  if (n < 1 || n > 64 || reserved != 0) return bad(why, "bad header");
  r.assign(n + 1, 0);
  if (fread(r.data(), 4, r.size(), f) != r.size()) return bad(why, "truncated header");
  if (r[0] != 1 || r[n] != 1) return bad(why, "bad boundary ranks");
  for (int k = 1; k < n; ++k)
    if (r[k] < 1 || r[k] > (1 << 20)) return bad(why, "bad bond rank");
  if (fseek(f, 0, SEEK_END) != 0) return bad(why, "seek failed");
  const long size = ftell(f);
  const size_t elems = payload_elems(r);  // < 2^47: no overflow for n <= 64, ranks <= 2^20
  if (size < 0 || (size_t)size != header_bytes(n) + 8 * elems)
    return bad(why, "file size disagrees with the bond ranks");
  if (fseek(f, (long)header_bytes(n), SEEK_SET) != 0) return bad(why, "seek failed");
  *n_out = n;
  *elems_out = elems;
  return VP_OK;
}

extern "C" int mps_file_info(const char* path, int* n_out, int* ranks_out, size_t* elems_out) {
  if (!path) return VP_EINVAL;
  File fh;
  fh.f = fopen(path, "rb");
  if (!fh.f) return VP_EIO;
  int n = 0;
  size_t elems = 0;
  std::vector<int> r;
  std::string why;
  VP_TRY(read_header(fh.f, &n, r, &elems, why));
  if (n_out) *n_out = n;
  if (ranks_out) std::copy(r.begin(), r.end(), ranks_out);
  if (elems_out) *elems_out = elems;
  return VP_OK;
}

extern "C" int mps_load(vp_ctx* ctx, const char* path, mps_t** out) {
  if (!ctx || !path || !out) return fail(ctx, VP_EINVAL, "mps_load: bad argument");
  *out = nullptr;
  File fh;
  fh.f = fopen(path, "rb");
  if (!fh.f) return fail(ctx, VP_EIO, std::string("mps_load: cannot open ") + path);
  int n = 0;
  size_t elems = 0;
  std::vector<int> r;
  std::string why;
  if (read_header(fh.f, &n, r, &elems, why) != VP_OK)
    return fail(ctx, VP_EIO, "mps_load: " + why + ": " + path);
  std::vector<double> cores;
  try {
    cores.resize(elems);
  } catch (const std::bad_alloc&) {
    return fail(ctx, VP_ENOMEM, "mps_load: host allocation failed");
  }
  if (fread(cores.data(), sizeof(double), cores.size(), fh.f) != cores.size())
    return fail(ctx, VP_EIO, "mps_load: truncated payload");
  return mps_create_cores(ctx, n, r.data(), cores.data(), out);
}
