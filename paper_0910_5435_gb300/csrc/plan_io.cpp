// plan_io.cpp -- plan files: the factorizations of a plan on disk.
//
// The precomputation of Section 3 (with the nodes of Section 4) dominates a
// plan's cold start, so a plan's factorizations can be written to a file and
// read back instead of recomputed.  The factor streams are not stored: they
// depend on run-time options (record chunk size, value cap, warps) and are
// re-encoded from the factorizations on load.
//
// File layout (little-endian, as the host writes it):
//   header (FileHeader, 128 bytes): magic, format version, the options that
//     determine the factorizations, the number of factorizations stored
//     (float64, then float32 if it was built), a hash of the unit table and a
//     hash of the header itself;
//   unit table: for each factorization and each parity block u = 2m + p, the
//     payload offset, size and hash of its serialized UnitFact;
//   payload: the serialized UnitFacts.
// Any mismatch (magic, version, sizes, a hash) is reported as PlanFileError.

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <memory>
#include <stdexcept>
#include <string>
#include <thread>
#include <vector>

#include <sys/types.h>  // off_t for fseeko / ftello

#include "plan_host.h"

namespace sht {
namespace {

constexpr char kMagic[8] = {'S', 'H', 'T', 'P', 'L', 'A', 'N', '\0'};
// 2: factorizations of the quadrature with exact-integer recurrence weights
// (version 1 files hold those of the earlier weights and are rebuilt)
constexpr uint32_t kVersion = 2;

struct FileHeader {
  char magic[8];
  uint32_t version;
  uint32_t nfact;  // 1: float64 factorizations; 2: float64 then float32
  int32_t l, leaf_cols, min_band_rows, units;
  double eps_id, trim_eps, eps_fp32;
  uint64_t table_hash;
  uint64_t header_hash;  // computed with this field zero
  uint8_t reserved[56];
};
static_assert(sizeof(FileHeader) == 128, "plan file header size");

struct UnitRecord {
  uint64_t offset, bytes, hash;
};

// 64-bit multiply-xorshift hash over 8-byte words (not cryptographic: it
// detects truncation and corruption).
uint64_t hash_bytes(const uint8_t* p, size_t n) {
  uint64_t h = 0x9E3779B97F4A7C15ull ^ (uint64_t)n;
  size_t i = 0;
  for (; i + 8 <= n; i += 8) {
    uint64_t w;
    std::memcpy(&w, p + i, 8);
    h = (h ^ w) * 0xFF51AFD7ED558CCDull;
    h ^= h >> 29;
  }
  uint64_t t = 0;
  if (i < n) std::memcpy(&t, p + i, n - i);
  h = (h ^ t) * 0xC4CEB9FE1A85EC53ull;
  h ^= h >> 32;
  return h;
}

struct Writer {
  std::vector<uint8_t> b;
  template <class T>
  void put(const T& v) {
    const uint8_t* p = reinterpret_cast<const uint8_t*>(&v);
    b.insert(b.end(), p, p + sizeof(T));
  }
  template <class T>
  void put_vec(const std::vector<T>& v) {
    put<uint64_t>(v.size());
    const uint8_t* p = reinterpret_cast<const uint8_t*>(v.data());
    b.insert(b.end(), p, p + sizeof(T) * v.size());
  }
};

struct Reader {
  const uint8_t* p;
  size_t n, at = 0;
  void need(size_t k) {
    if (k > n - at) throw PlanFileError("plan file: unit record ends early");
  }
  template <class T>
  T get() {
    need(sizeof(T));
    T v;
    std::memcpy(&v, p + at, sizeof(T));
    at += sizeof(T);
    return v;
  }
  template <class T>
  void get_vec(std::vector<T>& v, uint64_t max_count) {
    const uint64_t c = get<uint64_t>();
    if (c > max_count) throw PlanFileError("plan file: implausible array length");
    need(sizeof(T) * c);
    v.resize(c);
    std::memcpy(v.data(), p + at, sizeof(T) * c);
    at += sizeof(T) * c;
  }
};

void write_unit(const UnitFact& U, Writer& w) {
  w.put<int32_t>(U.m);
  w.put<int32_t>(U.p);
  w.put<int32_t>(U.n);
  w.put<int32_t>(U.rows);
  w.put<int32_t>(U.direct ? 1 : 0);
  w.put<int32_t>(U.levels);
  w.put<int64_t>(U.values);
  w.put<int64_t>(U.idx);
  w.put<int64_t>(U.peak_words);
  w.put<int64_t>(U.swaps);
  w.put<double>(U.cost);
  w.put_vec(U.D);
  w.put_vec(U.width);
  w.put<uint64_t>(U.blocks.size());
  for (const IdBlock& b : U.blocks) {
    const int32_t f[10] = {b.level, b.band, b.group, b.r0, b.r1, b.in_off, b.nin, b.k, b.out_off, 0};
    for (int32_t x : f) w.put(x);
    w.put_vec(b.skel);
    w.put_vec(b.red);
    w.put_vec(b.T);
  }
  w.put<uint64_t>(U.finals.size());
  for (const FinalBlock& f : U.finals) {
    const int32_t g[6] = {f.band, f.r0, f.r1, f.k, f.in_off, 0};
    for (int32_t x : g) w.put(x);
    w.put_vec(f.S);
  }
}

void read_unit(Reader& r, UnitFact& U, int l) {
  const uint64_t cap = (uint64_t)4 * l * l + 64;  // no array of a unit exceeds its dense block
  U.m = r.get<int32_t>();
  U.p = r.get<int32_t>();
  U.n = r.get<int32_t>();
  U.rows = r.get<int32_t>();
  U.direct = r.get<int32_t>() != 0;
  U.levels = r.get<int32_t>();
  U.values = r.get<int64_t>();
  U.idx = r.get<int64_t>();
  U.peak_words = r.get<int64_t>();
  U.swaps = r.get<int64_t>();
  U.cost = r.get<double>();
  r.get_vec(U.D, cap);
  r.get_vec(U.width, 64);
  // a serialized ID block is at least ten int32 fields and three array
  // lengths, a final block six int32 fields and one length: counts are bounded
  // by the bytes left in the record before anything is allocated for them
  constexpr uint64_t kMinBlockBytes = 10 * sizeof(int32_t) + 3 * sizeof(uint64_t);
  constexpr uint64_t kMinFinalBytes = 6 * sizeof(int32_t) + sizeof(uint64_t);
  const uint64_t nb = r.get<uint64_t>();
  if (nb > cap || nb > (r.n - r.at) / kMinBlockBytes) throw PlanFileError("plan file: implausible block count");
  U.blocks.resize(nb);
  for (IdBlock& b : U.blocks) {
    int32_t f[10];
    for (int32_t& x : f) x = r.get<int32_t>();
    b.level = f[0];
    b.band = f[1];
    b.group = f[2];
    b.r0 = f[3];
    b.r1 = f[4];
    b.in_off = f[5];
    b.nin = f[6];
    b.k = f[7];
    b.out_off = f[8];
    r.get_vec(b.skel, cap);
    r.get_vec(b.red, cap);
    r.get_vec(b.T, cap);
    if (b.k < 0 || b.nin < b.k || (int)b.skel.size() != b.k || (int)b.red.size() != b.nin - b.k ||
        b.T.size() != (size_t)b.k * (b.nin - b.k) || b.r0 < 0 || b.r1 < b.r0 || b.r1 > l)
      throw PlanFileError("plan file: inconsistent ID block");
    for (uint16_t s : b.skel)
      if (s >= b.nin) throw PlanFileError("plan file: skeleton index out of range");
    for (uint16_t s : b.red)
      if (s >= b.nin) throw PlanFileError("plan file: redundant index out of range");
  }
  const uint64_t nf = r.get<uint64_t>();
  if (nf > cap || nf > (r.n - r.at) / kMinFinalBytes) throw PlanFileError("plan file: implausible final block count");
  U.finals.resize(nf);
  for (FinalBlock& f : U.finals) {
    int32_t g[6];
    for (int32_t& x : g) x = r.get<int32_t>();
    f.band = g[0];
    f.r0 = g[1];
    f.r1 = g[2];
    f.k = g[3];
    f.in_off = g[4];
    r.get_vec(f.S, cap);
    if (f.k < 0 || f.r0 < 0 || f.r1 < f.r0 || f.r1 > l || f.S.size() != (size_t)(f.r1 - f.r0) * f.k)
      throw PlanFileError("plan file: inconsistent final block");
  }
  if (r.at != r.n) throw PlanFileError("plan file: unit record has trailing bytes");
  // the layout must index only inside the unit's vectors, whatever the file
  // says: the encoder turns these offsets into shared-memory positions
  const int L = 2 * l;
  if (U.m < 0 || U.m >= L || U.p < 0 || U.p > 1 || U.n != std::max(0, (L - U.m - U.p + 1) / 2) || U.rows < 0 ||
      U.rows > l || (U.direct && U.D.size() != (size_t)U.rows * U.n) || (!U.direct && !U.D.empty()))
    throw PlanFileError("plan file: inconsistent unit");
  const int lam = U.levels;
  const bool has_layout = !U.direct && U.n > 0 && U.rows > 0;
  if (!has_layout) {
    if (!U.blocks.empty() || !U.finals.empty()) throw PlanFileError("plan file: blocks in a unit without a butterfly");
    return;
  }
  if (lam < 0 || lam > 16 || (int)U.width.size() != lam + 2) throw PlanFileError("plan file: inconsistent levels");
  for (int j = 1; j <= lam + 1; ++j)
    if (U.width[j] < 0 || U.width[j] > 65535) throw PlanFileError("plan file: level width out of range");
  for (const IdBlock& b : U.blocks) {
    const int below = b.level == 1 ? U.n : (b.level >= 2 && b.level <= lam + 1 ? U.width[b.level - 1] : -1);
    if (b.level < 1 || b.level > lam + 1 || b.band < 0 || b.band >= (1 << (b.level - 1)) || b.group < 0 ||
        b.group >= (1 << (lam - b.level + 1)) || b.r0 >= b.r1 || b.r1 > U.rows || b.out_off < 0 ||
        b.out_off + b.k > U.width[b.level] || b.in_off < 0 || b.in_off + b.nin > below)
      throw PlanFileError("plan file: ID block outside its level's layout");
  }
  for (const FinalBlock& f : U.finals)
    if (f.band < 0 || f.band >= (1 << lam) || f.r0 >= f.r1 || f.r1 > U.rows || f.in_off < 0 ||
        f.in_off + f.k > U.width[lam + 1])
      throw PlanFileError("plan file: final block outside the top level's layout");
}

// Runs body(i) for i < count on the plan's host threads.
template <class F>
void parallel(int count, int threads, F&& body) {
  int nt = threads > 0 ? threads : (int)std::thread::hardware_concurrency();
  nt = std::max(1, std::min(nt, 256));
  std::atomic<int> next(0);
  std::vector<std::string> errors(nt);
  std::vector<int> corrupt(nt, 0);
  auto worker = [&](int tid) {
    try {
      for (;;) {
        const int i = next.fetch_add(1);
        if (i >= count) break;
        body(i);
      }
    } catch (const PlanFileError& e) {
      errors[tid] = e.what();
      corrupt[tid] = 1;
      next.store(count);
    } catch (const std::exception& e) {
      errors[tid] = e.what();
      next.store(count);
    }
  };
  std::vector<std::thread> th;
  for (int t = 1; t < nt; ++t) th.emplace_back(worker, t);
  worker(0);
  for (auto& t : th) t.join();
  for (int t = 0; t < nt; ++t)
    if (!errors[t].empty()) {
      if (corrupt[t]) throw PlanFileError(errors[t]);
      throw std::runtime_error(errors[t]);
    }
}

struct File {
  std::FILE* f = nullptr;
  ~File() {
    if (f) std::fclose(f);
  }
};

uint64_t header_hash(FileHeader h) {
  h.header_hash = 0;
  return hash_bytes(reinterpret_cast<const uint8_t*>(&h), sizeof h);
}

}  // namespace

void save_factorizations(const PlanHost& P, const std::string& path) {
  const int L = 2 * P.l, units = 2 * L;
  if ((int)P.fact64.size() != units) throw std::runtime_error("plan file: the plan has no float64 factorization");
  const bool with32 = (int)P.fact32.size() == units;
  const int nfact = with32 ? 2 : 1;
  std::vector<Writer> parts((size_t)nfact * units);
  std::vector<UnitRecord> table((size_t)nfact * units);
  parallel(nfact * units, P.num_threads, [&](int i) {
    const UnitFact& U = (i < units ? P.fact64 : P.fact32)[i % units];
    write_unit(U, parts[i]);
    table[i].bytes = parts[i].b.size();
    table[i].hash = hash_bytes(parts[i].b.data(), parts[i].b.size());
  });
  uint64_t off = 0;
  for (UnitRecord& r : table) {
    r.offset = off;
    off += r.bytes;
  }
  FileHeader h;
  std::memset(&h, 0, sizeof h);
  std::memcpy(h.magic, kMagic, 8);
  h.version = kVersion;
  h.nfact = (uint32_t)nfact;
  h.l = P.l;
  h.leaf_cols = P.leaf_cols;
  h.min_band_rows = P.min_band_rows;
  h.units = units;
  h.eps_id = P.eps_id;
  h.trim_eps = P.trim_eps;
  h.eps_fp32 = P.eps_fp32;
  h.table_hash = hash_bytes(reinterpret_cast<const uint8_t*>(table.data()), sizeof(UnitRecord) * table.size());
  h.header_hash = header_hash(h);
  // write to a temporary name, then rename: a crash leaves no half-written plan
  const std::string tmp = path + ".partial";
  {
    File f;
    f.f = std::fopen(tmp.c_str(), "wb");
    if (!f.f) throw std::runtime_error("plan file: cannot open " + tmp + " for writing");
    bool ok = std::fwrite(&h, sizeof h, 1, f.f) == 1 &&
              std::fwrite(table.data(), sizeof(UnitRecord), table.size(), f.f) == table.size();
    for (size_t i = 0; ok && i < parts.size(); ++i)
      ok = parts[i].b.empty() || std::fwrite(parts[i].b.data(), 1, parts[i].b.size(), f.f) == parts[i].b.size();
    ok = ok && std::fflush(f.f) == 0;
    if (!ok) {
      std::remove(tmp.c_str());
      throw std::runtime_error("plan file: write to " + tmp + " failed");
    }
  }
  if (std::rename(tmp.c_str(), path.c_str()) != 0) {
    std::remove(tmp.c_str());
    throw std::runtime_error("plan file: cannot rename " + tmp + " to " + path);
  }
}

bool read_plan_file_header(const std::string& path, PlanFileInfo* info) {
  File f;
  f.f = std::fopen(path.c_str(), "rb");
  if (!f.f) return false;
  FileHeader h;
  if (std::fread(&h, sizeof h, 1, f.f) != 1) throw PlanFileError("plan file: shorter than its header");
  if (std::memcmp(h.magic, kMagic, 8) != 0) throw PlanFileError("plan file: not a plan file (bad magic)");
  if (h.version != kVersion) throw PlanFileError("plan file: unsupported format version");
  if (header_hash(h) != h.header_hash) throw PlanFileError("plan file: header checksum mismatch");
  if (h.l < 1 || h.l > 1024 || h.units != 4 * h.l || h.nfact < 1 || h.nfact > 2)
    throw PlanFileError("plan file: implausible header");
  info->l = h.l;
  info->leaf_cols = h.leaf_cols;
  info->min_band_rows = h.min_band_rows;
  info->eps_id = h.eps_id;
  info->trim_eps = h.trim_eps;
  info->eps_fp32 = h.eps_fp32;
  info->has_fp32 = h.nfact == 2;
  return true;
}

void load_factorizations(PlanHost& P, const std::string& path) {
  File f;
  f.f = std::fopen(path.c_str(), "rb");
  if (!f.f) throw std::runtime_error("plan file: cannot open " + path);
  FileHeader h;
  if (std::fread(&h, sizeof h, 1, f.f) != 1) throw PlanFileError("plan file: shorter than its header");
  if (std::memcmp(h.magic, kMagic, 8) != 0) throw PlanFileError("plan file: not a plan file (bad magic)");
  if (h.version != kVersion) throw PlanFileError("plan file: unsupported format version");
  if (header_hash(h) != h.header_hash) throw PlanFileError("plan file: header checksum mismatch");
  if (h.l != P.l || h.units != 4 * P.l || h.nfact < 1 || h.nfact > 2)
    throw PlanFileError("plan file: header does not match the plan");
  const size_t nrec = (size_t)h.nfact * h.units;
  std::vector<UnitRecord> table(nrec);
  if (std::fread(table.data(), sizeof(UnitRecord), nrec, f.f) != nrec)
    throw PlanFileError("plan file: unit table ends early");
  if (hash_bytes(reinterpret_cast<const uint8_t*>(table.data()), sizeof(UnitRecord) * nrec) != h.table_hash)
    throw PlanFileError("plan file: unit table checksum mismatch");
  // The payload is the rest of the file.  Every record must fit in what is
  // left of it, so that a forged table (its hash is not cryptographic) can
  // neither wrap the running sum nor size an allocation beyond the file.
  const off_t here = ftello(f.f);
  if (here < 0 || fseeko(f.f, 0, SEEK_END) != 0) throw PlanFileError("plan file: cannot determine its size");
  const off_t end = ftello(f.f);
  if (end < here || fseeko(f.f, here, SEEK_SET) != 0) throw PlanFileError("plan file: cannot determine its size");
  const uint64_t avail = (uint64_t)(end - here);
  uint64_t total = 0;
  for (const UnitRecord& r : table) {
    if (r.offset != total) throw PlanFileError("plan file: unit table is not contiguous");
    if (r.bytes > avail - total) throw PlanFileError("plan file: payload ends early");
    total += r.bytes;
  }
  if (total != avail) throw PlanFileError("plan file: trailing bytes after the payload");
  ByteBuf payload;
  payload.resize(total);
  if (total && std::fread(payload.data(), 1, total, f.f) != total) throw PlanFileError("plan file: payload ends early");
  if (std::fgetc(f.f) != EOF) throw PlanFileError("plan file: trailing bytes after the payload");
  const int units = h.units;
  std::vector<UnitFact> f64(units), f32(h.nfact == 2 ? units : 0);
  parallel((int)nrec, P.num_threads, [&](int i) {
    const UnitRecord& r = table[i];
    const uint8_t* p = payload.data() + r.offset;
    if (hash_bytes(p, r.bytes) != r.hash) throw PlanFileError("plan file: unit checksum mismatch");
    Reader rd{p, r.bytes};
    UnitFact& U = (i < units ? f64 : f32)[i % units];
    read_unit(rd, U, P.l);
    if (U.m != (i % units) / 2 || U.p != (i % units) % 2) throw PlanFileError("plan file: units out of order");
  });
  P.fact64.swap(f64);
  P.fact32.swap(f32);
}

}  // namespace sht
