// fr_h5.cpp -- host-side HDF5 drain of finished maps and scalar features
// (the paper's "Structured HDF5 storage": one file per extraction holding the
// results with the image and mask arrays, the voxel geometry, the extraction
// settings and an identification of the input; scalar results as ordered
// feature names and float64 values, spatial results as named maps with their
// source geometry; LZF or gzip compression chosen in the settings).
//
// The file is written directly in the HDF5 format (superblock version 0,
// version-1 object headers, symbol-table groups, chunked datasets indexed by
// a version-1 B-tree, filter pipeline deflate / shuffle / LZF), so no HDF5
// library is needed at build or run time.  Chunks are scattered from the
// compact [rows][n_voi] maps and compressed on a pool of host threads; a map
// chunk that holds no VOI voxel is not stored at all and reads back as the
// dataset's fill value (NaN).  gzip uses the system zlib, loaded with dlopen.
#include <dlfcn.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <ctime>
#include <limits>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "flashmap.h"

namespace {

constexpr uint64_t kUndef = ~0ull;
constexpr int kGroupLeafK = 4;       // symbol-table node: up to 2K entries
constexpr int kGroupInternalK = 16;  // group B-tree node: up to 2K children
constexpr int kChunkK = 32;          // chunk B-tree node: up to 2K children
constexpr int kMaxChunks = 2 * kChunkK;
constexpr int32_t kAutoChunk[3] = {0, 0, 0};

// ------------------------------------------------------------------ bytes
struct Bytes {
  std::vector<uint8_t> b;
  void u8(unsigned v) { b.push_back((uint8_t)v); }
  void u16(unsigned v) { u8(v & 0xFF), u8((v >> 8) & 0xFF); }
  void u32(uint32_t v) {
    for (int i = 0; i < 4; ++i) u8((v >> (8 * i)) & 0xFF);
  }
  void u64(uint64_t v) {
    for (int i = 0; i < 8; ++i) u8((unsigned)((v >> (8 * i)) & 0xFF));
  }
  void raw(const void* p, size_t n) {
    const uint8_t* c = (const uint8_t*)p;
    b.insert(b.end(), c, c + n);
  }
  void zeros(size_t n) { b.insert(b.end(), n, 0); }
  void pad8() {
    while (b.size() % 8) u8(0);
  }
  size_t size() const { return b.size(); }
};

// ------------------------------------------------------------------- zlib
// The two zlib entry points used (zlib's documented C API; uLong is unsigned
// long on the LP64 targets this library builds for).
struct Zlib {
  using compress2_fn = int (*)(unsigned char*, unsigned long*, const unsigned char*,
                               unsigned long, int);
  using bound_fn = unsigned long (*)(unsigned long);
  compress2_fn compress2 = nullptr;
  bound_fn bound = nullptr;
  bool ok = false;
};

const Zlib& zlib() {
  static Zlib z;
  static std::once_flag once;
  std::call_once(once, [] {
    void* h = dlopen("libz.so.1", RTLD_NOW | RTLD_LOCAL);
    if (!h) h = dlopen("libz.so", RTLD_NOW | RTLD_LOCAL);
    if (!h) return;
    z.compress2 = (Zlib::compress2_fn)dlsym(h, "compress2");
    z.bound = (Zlib::bound_fn)dlsym(h, "compressBound");
    z.ok = z.compress2 && z.bound;
  });
  return z;
}

// -------------------------------------------------------------------- LZF
// LZF stream (liblzf's format): a control byte c < 32 introduces a literal
// run of c + 1 bytes; otherwise the top three bits give a match length
// L = c >> 5 (L == 7: plus the next byte), and (c & 31) << 8 | next byte is
// the distance minus one; L + 2 bytes are copied from that far back.  This
// compressor is greedy over a hash of 3-byte prefixes.  Returns the output
// size, or 0 when the output would not be smaller than the input.
size_t lzf_compress(const uint8_t* in, size_t n, uint8_t* out, size_t cap) {
  constexpr int kHashBits = 14;
  constexpr size_t kMaxOff = 1u << 13, kMaxLit = 32, kMaxRef = 264;
  std::vector<int64_t> table((size_t)1 << kHashBits, -1);
  size_t ip = 0, op = 0, lit_start = 0;
  auto flush_lits = [&](size_t end) -> bool {
    size_t p = lit_start;
    while (p < end) {
      const size_t run = std::min(kMaxLit, end - p);
      if (op + 1 + run > cap) return false;
      out[op++] = (uint8_t)(run - 1);
      std::memcpy(out + op, in + p, run);
      op += run;
      p += run;
    }
    return true;
  };
  while (ip + 2 < n) {
    const uint32_t key = ((uint32_t)in[ip] << 16) | ((uint32_t)in[ip + 1] << 8) | in[ip + 2];
    const uint32_t h = (key * 2654435761u) >> (32 - kHashBits);
    const int64_t ref = table[h];
    table[h] = (int64_t)ip;
    if (ref >= 0 && ip - (size_t)ref <= kMaxOff && in[ref] == in[ip] &&
        in[ref + 1] == in[ip + 1] && in[ref + 2] == in[ip + 2]) {
      size_t len = 3;
      while (len < kMaxRef && ip + len < n && in[ref + len] == in[ip + len]) ++len;
      if (!flush_lits(ip)) return 0;
      const size_t off = ip - (size_t)ref - 1, l = len - 2;
      if (op + 3 > cap) return 0;
      if (l < 7) {
        out[op++] = (uint8_t)((l << 5) | (off >> 8));
      } else {
        out[op++] = (uint8_t)((7 << 5) | (off >> 8));
        out[op++] = (uint8_t)(l - 7);
      }
      out[op++] = (uint8_t)(off & 0xFF);
      ip += len;
      lit_start = ip;
      continue;
    }
    ++ip;
  }
  if (!flush_lits(n)) return 0;
  return op < n ? op : 0;
}

// ----------------------------------------------------------- dataset plan
enum DType { kI16, kU8, kF32, kF64, kI64, kStr };

size_t dtype_size(DType t, size_t strlen_) {
  switch (t) {
    case kI16: return 2;
    case kU8: return 1;
    case kF32: return 4;
    case kF64: return 8;
    case kI64: return 8;
    default: return strlen_;
  }
}

// datatype message (version 1)
void put_datatype(Bytes& o, DType t, size_t str_size) {
  switch (t) {
    case kF32:
    case kF64: {
      const bool d = t == kF64;
      o.u8(0x11);  // version 1, class 1 (floating point)
      o.u8(0x20);  // little endian, implied leading mantissa bit
      o.u8(d ? 63 : 31);  // sign bit position
      o.u8(0);
      o.u32(d ? 8 : 4);
      o.u16(0);
      o.u16(d ? 64 : 32);
      o.u8(d ? 52 : 23);  // exponent location
      o.u8(d ? 11 : 8);   // exponent size
      o.u8(0);            // mantissa location
      o.u8(d ? 52 : 23);  // mantissa size
      o.u32(d ? 1023 : 127);
      break;
    }
    case kI16:
    case kU8:
    case kI64: {
      const size_t n = dtype_size(t, 0);
      o.u8(0x10);                     // version 1, class 0 (fixed point)
      o.u8(t == kU8 ? 0x00 : 0x08);   // little endian, signed unless u8
      o.u8(0);
      o.u8(0);
      o.u32((uint32_t)n);
      o.u16(0);
      o.u16((unsigned)(8 * n));
      break;
    }
    case kStr:
      o.u8(0x13);  // version 1, class 3 (string)
      o.u8(0x00);  // null terminated, ASCII
      o.u8(0);
      o.u8(0);
      o.u32((uint32_t)str_size);
      break;
  }
}

void put_dataspace(Bytes& o, const std::vector<uint64_t>& dims) {
  o.u8(1);
  o.u8((unsigned)dims.size());
  o.u8(0);  // no maximum dimensions: fixed size
  o.u8(0);
  o.u32(0);
  for (uint64_t d : dims) o.u64(d);
}

struct Attr {
  std::string name;
  DType t;
  std::vector<double> f;
  std::vector<int64_t> i;
  std::string s;
};

Attr attr_f64(const std::string& n, std::vector<double> v) { return Attr{n, kF64, v, {}, {}}; }
Attr attr_i64(const std::string& n, std::vector<int64_t> v) { return Attr{n, kI64, {}, v, {}}; }
Attr attr_str(const std::string& n, const std::string& s) { return Attr{n, kStr, {}, {}, s}; }

// attribute message (version 1): name, datatype and dataspace each padded to 8
void put_attribute(Bytes& o, const Attr& a) {
  Bytes dt, ds, data;
  size_t n = 1;
  if (a.t == kStr) {
    put_datatype(dt, kStr, a.s.size() + 1);
    data.raw(a.s.c_str(), a.s.size() + 1);
  } else if (a.t == kF64) {
    put_datatype(dt, kF64, 0);
    n = a.f.size();
    for (double v : a.f) data.raw(&v, 8);
  } else {
    put_datatype(dt, kI64, 0);
    n = a.i.size();
    for (int64_t v : a.i) data.raw(&v, 8);
  }
  put_dataspace(ds, {(uint64_t)n});
  o.u8(1);
  o.u8(0);
  o.u16((unsigned)(a.name.size() + 1));
  o.u16((unsigned)dt.size());
  o.u16((unsigned)ds.size());
  o.raw(a.name.c_str(), a.name.size() + 1);
  o.pad8();
  o.raw(dt.b.data(), dt.size());
  o.pad8();
  o.raw(ds.b.data(), ds.size());
  o.pad8();
  o.raw(data.b.data(), data.size());
}

// one header message: type, size, flags, then the body padded to 8
void put_message(Bytes& o, unsigned type, const Bytes& body, unsigned flags = 0) {
  Bytes b = body;
  b.pad8();
  o.u16(type);
  o.u16((unsigned)b.size());
  o.u8(flags);
  o.u8(0);
  o.u8(0);
  o.u8(0);
  o.raw(b.b.data(), b.size());
}

// version-1 object header around its messages
Bytes object_header(const std::vector<Bytes>& msgs) {
  Bytes body;
  for (const Bytes& m : msgs) body.raw(m.b.data(), m.size());
  Bytes o;
  o.u8(1);
  o.u8(0);
  o.u16((unsigned)msgs.size());
  o.u32(1);  // reference count
  o.u32((uint32_t)body.size());
  o.u32(0);  // pad the 12-byte prefix to 16
  o.raw(body.b.data(), body.size());
  return o;
}

// ------------------------------------------------------------------ file
class Writer {
 public:
  explicit Writer(FILE* f) : f_(f) {
    Bytes zero;
    zero.zeros(96);  // superblock, written last
    put(zero);
  }
  uint64_t put(const Bytes& b) {
    const uint64_t at = pos_;
    if (b.size() && std::fwrite(b.b.data(), 1, b.size(), f_) != b.size()) ok_ = false;
    pos_ += b.size();
    if (pos_ % 8) {  // keep every structure 8-byte aligned
      Bytes p;
      p.zeros(8 - pos_ % 8);
      if (std::fwrite(p.b.data(), 1, p.size(), f_) != p.size()) ok_ = false;
      pos_ += p.size();
    }
    return at;
  }
  uint64_t put_raw(const void* p, size_t n) {
    Bytes b;
    b.raw(p, n);
    return put(b);
  }
  bool finish(uint64_t root_header, uint64_t root_btree, uint64_t root_heap) {
    Bytes s;
    const uint8_t sig[8] = {0x89, 'H', 'D', 'F', '\r', '\n', 0x1a, '\n'};
    s.raw(sig, 8);
    s.u8(0), s.u8(0), s.u8(0), s.u8(0), s.u8(0);  // versions
    s.u8(8), s.u8(8), s.u8(0);                    // offset / length sizes
    s.u16(kGroupLeafK);
    s.u16(kGroupInternalK);
    s.u32(0);       // consistency flags
    s.u64(0);       // base address
    s.u64(kUndef);  // free-space info
    s.u64(pos_);    // end of file
    s.u64(kUndef);  // driver information
    // root group symbol table entry
    s.u64(0);
    s.u64(root_header);
    s.u32(1);  // cache type 1: B-tree and heap addresses follow
    s.u32(0);
    s.u64(root_btree);
    s.u64(root_heap);
    if (std::fseek(f_, 0, SEEK_SET) != 0) return false;
    if (std::fwrite(s.b.data(), 1, s.size(), f_) != s.size()) return false;
    return ok_;
  }
  bool ok() const { return ok_; }

 private:
  FILE* f_;
  uint64_t pos_ = 0;
  bool ok_ = true;
};

struct Link {
  std::string name;
  uint64_t header;
  bool group;
  uint64_t btree, heap;  // groups: cached in the symbol table entry
};

struct GroupAddr {
  uint64_t header, btree, heap;
};

// A symbol-table group: local heap of names, symbol-table nodes of at most
// 2 * kGroupLeafK sorted entries, one B-tree node over them, object header.
bool write_group(Writer& w, std::vector<Link> links, const std::vector<Attr>& attrs,
                 GroupAddr* out) {
  std::sort(links.begin(), links.end(),
            [](const Link& a, const Link& b) { return std::strcmp(a.name.c_str(), b.name.c_str()) < 0; });
  const size_t per_node = 2 * kGroupLeafK;
  const size_t nodes = (links.size() + per_node - 1) / per_node;
  if (nodes > 2 * (size_t)kGroupInternalK) return false;
  // heap data: "" at 0, then each name (null terminated, padded to 8)
  Bytes hd;
  hd.zeros(8);
  std::vector<uint64_t> name_off(links.size());
  for (size_t k = 0; k < links.size(); ++k) {
    name_off[k] = hd.size();
    hd.raw(links[k].name.c_str(), links[k].name.size() + 1);
    hd.pad8();
  }
  const uint64_t hdata = w.put(hd);
  Bytes heap;
  heap.raw("HEAP", 4);
  heap.u8(0), heap.u8(0), heap.u8(0), heap.u8(0);
  heap.u64(hd.size());
  heap.u64(1);  // no free block (the HDF5 library ends its free list with 1)
  heap.u64(hdata);
  const uint64_t heap_addr = w.put(heap);
  std::vector<uint64_t> snod(nodes);
  for (size_t n = 0; n < nodes; ++n) {
    Bytes s;
    s.raw("SNOD", 4);
    s.u8(1);
    s.u8(0);
    const size_t k0 = n * per_node, k1 = std::min(links.size(), k0 + per_node);
    s.u16((unsigned)(k1 - k0));
    for (size_t k = k0; k < k1; ++k) {
      s.u64(name_off[k]);
      s.u64(links[k].header);
      s.u32(links[k].group ? 1 : 0);
      s.u32(0);
      if (links[k].group) {
        s.u64(links[k].btree);
        s.u64(links[k].heap);
      } else {
        s.zeros(16);
      }
    }
    s.zeros(40 * (per_node - (k1 - k0)));
    snod[n] = w.put(s);
  }
  Bytes t;
  t.raw("TREE", 4);
  t.u8(0);  // group node
  t.u8(0);  // leaf level
  t.u16((unsigned)nodes);
  t.u64(kUndef);
  t.u64(kUndef);
  t.u64(0);  // key 0: the empty name
  for (size_t n = 0; n < nodes; ++n) {
    const size_t last = std::min(links.size(), (n + 1) * per_node) - 1;
    t.u64(snod[n]);
    t.u64(name_off[last]);
  }
  const size_t full = 24 + (2 * kGroupInternalK) * 8 + (2 * kGroupInternalK + 1) * 8;
  t.zeros(full - t.size());
  const uint64_t btree = w.put(t);
  std::vector<Bytes> msgs;
  Bytes st;
  st.u64(btree);
  st.u64(heap_addr);
  Bytes m;
  put_message(m, 0x11, st);
  msgs.push_back(m);
  for (const Attr& a : attrs) {
    Bytes body, mm;
    put_attribute(body, a);
    put_message(mm, 0x0C, body);
    msgs.push_back(mm);
  }
  out->header = w.put(object_header(msgs));
  out->btree = btree;
  out->heap = heap_addr;
  return w.ok();
}

// Contiguous dataset (small arrays: feature names and values).
uint64_t write_contiguous(Writer& w, DType t, size_t str_size, const std::vector<uint64_t>& dims,
                          const void* data, size_t bytes, const std::vector<Attr>& attrs) {
  const uint64_t at = w.put_raw(data, bytes);
  std::vector<Bytes> msgs;
  Bytes b, m;
  put_dataspace(b, dims);
  put_message(m, 0x01, b);
  msgs.push_back(m);
  b = Bytes(), m = Bytes();
  put_datatype(b, t, str_size);
  put_message(m, 0x03, b, 1);
  msgs.push_back(m);
  b = Bytes(), m = Bytes();
  b.u8(2), b.u8(2), b.u8(2), b.u8(0);  // fill value v2: late, if set, undefined
  put_message(m, 0x05, b, 1);
  msgs.push_back(m);
  b = Bytes(), m = Bytes();
  b.u8(3), b.u8(1);  // layout version 3, contiguous
  b.u64(at);
  b.u64(bytes);
  put_message(m, 0x08, b);
  msgs.push_back(m);
  for (const Attr& a : attrs) {
    Bytes body, mm;
    put_attribute(body, a);
    put_message(mm, 0x0C, body);
    msgs.push_back(mm);
  }
  return w.put(object_header(msgs));
}

struct Codec {
  int codec, level, shuffle, threads;
};

// One stored chunk: its offsets in the dataset, filter mask and bytes.
struct Chunk {
  uint64_t off[3];
  uint32_t mask = 0;
  std::vector<uint8_t> bytes;
  bool present = false;
};

// Shuffle (HDF5 filter 2): byte k of every element, element after element,
// for k = 0 .. size-1.
void shuffle_bytes(const std::vector<uint8_t>& in, size_t es, std::vector<uint8_t>& out) {
  const size_t n = in.size() / es;
  out.resize(in.size());
  for (size_t k = 0; k < es; ++k)
    for (size_t e = 0; e < n; ++e) out[k * n + e] = in[e * es + k];
}

// Apply the pipeline to one raw chunk.  Mandatory filters (shuffle, deflate)
// always apply; LZF is optional and is skipped (mask bit) when it does not
// shrink the chunk.
bool encode_chunk(const Codec& c, size_t es, std::vector<uint8_t>& raw, Chunk& ch) {
  std::vector<uint8_t> buf;
  int fi = 0;
  if (c.shuffle && es > 1) {
    shuffle_bytes(raw, es, buf);
    raw.swap(buf);
    ++fi;
  }
  if (c.codec == FR_H5_GZIP) {
    const Zlib& z = zlib();
    unsigned long cap = z.bound((unsigned long)raw.size());
    buf.resize(cap);
    if (z.compress2(buf.data(), &cap, raw.data(), (unsigned long)raw.size(), c.level) != 0)
      return false;
    buf.resize(cap);
    ch.bytes.swap(buf);
  } else if (c.codec == FR_H5_LZF) {
    buf.resize(raw.size());
    const size_t n = lzf_compress(raw.data(), raw.size(), buf.data(), buf.size());
    if (n) {
      buf.resize(n);
      ch.bytes.swap(buf);
    } else {
      ch.mask |= 1u << fi;
      ch.bytes.swap(raw);
    }
  } else {
    ch.bytes.swap(raw);
  }
  ch.present = true;
  return true;
}

void put_filters(std::vector<Bytes>& msgs, const Codec& c, size_t es, size_t chunk_bytes) {
  struct F {
    unsigned id, flags;
    std::string name;
    std::vector<uint32_t> cd;
  };
  std::vector<F> fs;
  if (c.shuffle && es > 1) fs.push_back({2, 0, "", {(uint32_t)es}});
  if (c.codec == FR_H5_GZIP) fs.push_back({1, 0, "", {(uint32_t)c.level}});
  // LZF (filter id 32000, as registered for h5py): optional; client data
  // filter revision, LZF version, chunk bytes (the decoder's buffer hint)
  if (c.codec == FR_H5_LZF) fs.push_back({32000, 1, "lzf", {4u, 0x0105u, (uint32_t)chunk_bytes}});
  if (fs.empty()) return;
  Bytes b;
  b.u8(1);
  b.u8((unsigned)fs.size());
  b.zeros(6);
  for (const F& f : fs) {
    const size_t nl = f.name.empty() ? 0 : f.name.size() + 1;
    b.u16(f.id);
    b.u16((unsigned)((nl + 7) & ~(size_t)7));
    b.u16(f.flags);
    b.u16((unsigned)f.cd.size());
    if (nl) {
      b.raw(f.name.c_str(), nl);
      b.pad8();
    }
    for (uint32_t v : f.cd) b.u32(v);
    if (f.cd.size() % 2) b.u32(0);
  }
  Bytes m;
  put_message(m, 0x0B, b, 1);
  msgs.push_back(m);
}

// Chunked 3-D dataset: stored chunks, one B-tree node indexing them (chunk
// keys: stored size, filter mask, offsets incl. the element dimension; the
// last key bounds the last chunk), then the object header.
uint64_t write_chunked(Writer& w, DType t, const uint64_t dims[3], const uint64_t cdim[3],
                       std::vector<Chunk>& chunks, const Codec& c, const void* fill,
                       const std::vector<Attr>& attrs) {
  const size_t es = dtype_size(t, 0);
  Bytes tb;
  tb.raw("TREE", 4);
  tb.u8(1);  // raw data chunk node
  tb.u8(0);  // leaf level
  size_t used = 0;
  const Chunk* last = nullptr;
  Bytes entries;
  for (Chunk& ch : chunks) {  // chunks are in row-major chunk-grid order
    if (!ch.present) continue;
    const uint64_t at = w.put_raw(ch.bytes.data(), ch.bytes.size());
    entries.u32((uint32_t)ch.bytes.size());
    entries.u32(ch.mask);
    entries.u64(ch.off[0]);
    entries.u64(ch.off[1]);
    entries.u64(ch.off[2]);
    entries.u64(0);
    entries.u64(at);
    std::vector<uint8_t>().swap(ch.bytes);
    ++used;
    last = &ch;
  }
  uint64_t btree = kUndef;
  if (used) {
    tb.u16((unsigned)used);
    tb.u64(kUndef);
    tb.u64(kUndef);
    tb.raw(entries.b.data(), entries.size());
    tb.u32(0);
    tb.u32(0);
    for (int d = 0; d < 3; ++d) tb.u64(last->off[d] + cdim[d]);
    tb.u64(es);
    const size_t key = 8 + 8 * 4;
    const size_t full = 24 + (2 * kChunkK) * 8 + (2 * kChunkK + 1) * key;
    tb.zeros(full - tb.size());
    btree = w.put(tb);
  }
  std::vector<Bytes> msgs;
  Bytes b, m;
  put_dataspace(b, {dims[0], dims[1], dims[2]});
  put_message(m, 0x01, b);
  msgs.push_back(m);
  b = Bytes(), m = Bytes();
  put_datatype(b, t, 0);
  put_message(m, 0x03, b, 1);
  msgs.push_back(m);
  b = Bytes(), m = Bytes();
  b.u8(2), b.u8(3), b.u8(2), b.u8(1);  // fill value v2: incremental, if set, defined
  b.u32((uint32_t)es);
  b.raw(fill, es);
  put_message(m, 0x05, b, 1);
  msgs.push_back(m);
  b = Bytes(), m = Bytes();
  b.u8(3), b.u8(2), b.u8(4);  // layout version 3, chunked, rank + 1
  b.u64(btree);
  for (int d = 0; d < 3; ++d) b.u32((uint32_t)cdim[d]);
  b.u32((uint32_t)es);
  put_message(m, 0x08, b);
  msgs.push_back(m);
  put_filters(msgs, c, es, (size_t)(cdim[0] * cdim[1] * cdim[2]) * es);
  for (const Attr& a : attrs) {
    Bytes body, mm;
    put_attribute(body, a);
    put_message(mm, 0x0C, body);
    msgs.push_back(mm);
  }
  return w.put(object_header(msgs));
}

// Chunk grid of a [nz][ny][nx] volume: the requested extents (0: a quarter
// of the volume), clamped to the volume, grown until at most kMaxChunks
// chunks (one B-tree node indexes them).
void chunk_grid(const int32_t req[3], const uint64_t dims[3], uint64_t cdim[3], uint64_t ng[3]) {
  for (int d = 0; d < 3; ++d) {
    uint64_t c = req[d] > 0 ? (uint64_t)req[d] : (dims[d] + 3) / 4;
    cdim[d] = std::max<uint64_t>(1, std::min<uint64_t>(c, dims[d]));
  }
  while (true) {
    for (int d = 0; d < 3; ++d) ng[d] = (dims[d] + cdim[d] - 1) / cdim[d];
    if (ng[0] * ng[1] * ng[2] <= (uint64_t)kMaxChunks) break;
    int g = 0;  // grow the dimension with the most chunks
    for (int d = 1; d < 3; ++d)
      if (ng[d] > ng[g]) g = d;
    cdim[g] = std::min<uint64_t>(dims[g], cdim[g] * 2);
  }
}

// Run task(k) for k in [0, n) on up to `threads` host threads.
template <class F>
bool parallel_for(size_t n, int threads, F task) {
  int nt = threads > 0 ? threads : (int)std::thread::hardware_concurrency();
  nt = std::max(1, std::min<int>(nt, (int)n));
  std::atomic<size_t> next{0};
  std::atomic<bool> ok{true};
  auto body = [&] {
    for (size_t k; (k = next.fetch_add(1)) < n;)
      if (!task(k)) ok = false;
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < nt; ++t) pool.emplace_back(body);
  body();
  for (auto& th : pool) th.join();
  return ok;
}

// Chunks of a host volume (image or mask), encoded in parallel.
template <class T>
bool volume_chunks(const T* v, const uint64_t dims[3], const uint64_t cdim[3],
                   const uint64_t ng[3], const Codec& c, std::vector<Chunk>& out) {
  out.assign(ng[0] * ng[1] * ng[2], Chunk());
  return parallel_for(out.size(), c.threads, [&](size_t k) {
    Chunk& ch = out[k];
    const uint64_t gz = k / (ng[1] * ng[2]), gy = (k / ng[2]) % ng[1], gx = k % ng[2];
    ch.off[0] = gz * cdim[0], ch.off[1] = gy * cdim[1], ch.off[2] = gx * cdim[2];
    std::vector<uint8_t> raw(cdim[0] * cdim[1] * cdim[2] * sizeof(T), 0);
    T* r = (T*)raw.data();
    for (uint64_t z = 0; z < cdim[0] && ch.off[0] + z < dims[0]; ++z)
      for (uint64_t y = 0; y < cdim[1] && ch.off[1] + y < dims[1]; ++y) {
        const uint64_t src = ((ch.off[0] + z) * dims[1] + ch.off[1] + y) * dims[2] + ch.off[2];
        const uint64_t n = std::min<uint64_t>(cdim[2], dims[2] - ch.off[2]);
        std::memcpy(r + (z * cdim[1] + y) * cdim[2], v + src, n * sizeof(T));
      }
    return encode_chunk(c, sizeof(T), raw, ch);
  });
}

std::string now_utc() {
  const std::time_t t = std::time(nullptr);
  std::tm g;
  gmtime_r(&t, &g);
  char buf[32];
  std::strftime(buf, sizeof buf, "%Y-%m-%dT%H:%M:%SZ", &g);
  return buf;
}

// Root attributes: geometry, settings and provenance of the extraction.
std::vector<Attr> root_attrs(const fr_map_params* p, const fr_h5_source* src, const char* mode,
                             const std::vector<int64_t>& ids) {
  std::vector<Attr> a;
  a.push_back(attr_str("format", "flashmap radiomics extraction"));
  a.push_back(attr_str("mode", mode));
  a.push_back(attr_i64("shape_zyx", {p->nz, p->ny, p->nx}));
  a.push_back(attr_f64("spacing_xyz_mm", {p->spacing[0], p->spacing[1], p->spacing[2]}));
  a.push_back(attr_f64("origin_xyz_mm", {src->origin[0], src->origin[1], src->origin[2]}));
  a.push_back(attr_str("discretisation", p->disc_mode == FR_FBN ? "FBN" : "FBW"));
  a.push_back(attr_i64("bin_count", {p->bin_count}));
  a.push_back(attr_f64("bin_width", {p->bin_width}));
  a.push_back(attr_str("fbw_anchor", p->fbw_anchor == FR_ANCHOR_ZERO_FLOOR ? "zero_floor" : "voi_min"));
  a.push_back(attr_i64("kernel_radius", {p->kernel_radius}));
  a.push_back(attr_i64("glcm_distance", {p->glcm_distance}));
  a.push_back(attr_str("aggregation", p->aggregation == FR_AGG_MERGED ? "merged" : "average"));
  a.push_back(attr_i64("kurtosis_excess", {p->kurtosis_excess}));
  a.push_back(attr_i64("feature_ids", ids));
  a.push_back(attr_str("source", src->source_id ? src->source_id : ""));
  a.push_back(attr_str("created_utc", now_utc()));
  a.push_back(attr_str("writer", "flashmap fr_h5"));
  return a;
}

std::vector<int64_t> selected_ids(const fr_map_params* p, int nfeat) {
  std::vector<int64_t> ids;
  for (int f = 0; f < nfeat; ++f)
    if ((p->feature_mask[f >> 6] >> (f & 63)) & 1ull) ids.push_back(f);
  return ids;
}

bool check_common(const char* path, const fr_map_params* p, const fr_h5_source* src,
                  const fr_h5_options* opt, Codec* c) {
  if (!path || !p || !src || !src->image || !src->mask) return false;
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return false;
  Codec d{FR_H5_GZIP, 4, 1, 0};
  if (opt) d = Codec{opt->codec, opt->level ? opt->level : 4, opt->shuffle, opt->threads};
  if (d.codec < FR_H5_NONE || d.codec > FR_H5_LZF || d.level < 1 || d.level > 9) return false;
  *c = d;
  return true;
}

}  // namespace

extern "C" {

fr_status fr_h5_options_init(fr_h5_options* o) {
  if (!o) return FR_ERR_INVALID_ARG;
  std::memset(o, 0, sizeof *o);
  o->codec = FR_H5_GZIP;
  o->level = 4;
  o->shuffle = 1;
  return FR_OK;
}

fr_status fr_h5_write_maps(const char* path, const fr_map_params* p, const fr_h5_source* src,
                           const float* maps, int32_t n_rows, int64_t n_voi,
                           const int32_t* voxel_index, const fr_h5_options* opt) {
  Codec c;
  if (!check_common(path, p, src, opt, &c) || !maps || !voxel_index || n_voi < 1)
    return FR_ERR_INVALID_ARG;
  const std::vector<int64_t> ids = selected_ids(p, FR_NUM_FEATURES);
  if ((int32_t)ids.size() != n_rows || n_rows < 1) return FR_ERR_INVALID_ARG;
  if (c.codec == FR_H5_GZIP && !zlib().ok) return FR_ERR_UNSUPPORTED;
  const uint64_t dims[3] = {(uint64_t)p->nz, (uint64_t)p->ny, (uint64_t)p->nx};
  const uint64_t nvox = dims[0] * dims[1] * dims[2];
  // dense column of every voxel (-1 outside the VOI)
  std::vector<int32_t> col;
  try {
    col.assign(nvox, -1);
  } catch (...) {
    return FR_ERR_OOM;
  }
  for (int64_t k = 0; k < n_voi; ++k) {
    const int64_t v = voxel_index[k];
    if (v < 0 || (uint64_t)v >= nvox) return FR_ERR_INVALID_ARG;
    col[v] = (int32_t)k;
  }
  uint64_t cdim[3], ng[3];
  chunk_grid(opt ? opt->chunk : kAutoChunk, dims, cdim, ng);
  const size_t nch = ng[0] * ng[1] * ng[2];
  FILE* f = std::fopen(path, "wb");
  if (!f) return FR_ERR_IO;
  Writer w(f);
  bool ok = true;
  std::vector<Link> root;
  try {
    std::vector<Chunk> ch;
    ok = ok && volume_chunks(src->image, dims, cdim, ng, c, ch);
    const int16_t fi = 0;
    const uint8_t fu = 0;
    if (ok)
      root.push_back({"image", write_chunked(w, kI16, dims, cdim, ch, c, &fi,
                                             {attr_str("unit", "stored intensity")}),
                      false, 0, 0});
    ok = ok && volume_chunks(src->mask, dims, cdim, ng, c, ch);
    if (ok) root.push_back({"mask", write_chunked(w, kU8, dims, cdim, ch, c, &fu, {}), false, 0, 0});
    // maps: [rows][chunks] encoded in parallel, written row by row
    std::vector<Link> maps_links;
    const float fnan = std::numeric_limits<float>::quiet_NaN();
    const int rows_per_pass = std::max(1, (int)(256 / std::max<size_t>(1, nch)));
    for (int r0 = 0; ok && r0 < n_rows; r0 += rows_per_pass) {
      const int r1 = std::min(n_rows, r0 + rows_per_pass);
      std::vector<std::vector<Chunk>> rc(r1 - r0, std::vector<Chunk>(nch));
      ok = parallel_for((size_t)(r1 - r0) * nch, c.threads, [&](size_t t) {
        const int r = r0 + (int)(t / nch);
        const size_t k = t % nch;
        Chunk& chk = rc[r - r0][k];
        const uint64_t gz = k / (ng[1] * ng[2]), gy = (k / ng[2]) % ng[1], gx = k % ng[2];
        chk.off[0] = gz * cdim[0], chk.off[1] = gy * cdim[1], chk.off[2] = gx * cdim[2];
        std::vector<uint8_t> raw(cdim[0] * cdim[1] * cdim[2] * 4);
        float* o = (float*)raw.data();
        const float* row = maps + (size_t)r * (size_t)n_voi;
        bool any = false;
        for (uint64_t z = 0; z < cdim[0]; ++z)
          for (uint64_t y = 0; y < cdim[1]; ++y)
            for (uint64_t x = 0; x < cdim[2]; ++x) {
              const uint64_t Z = chk.off[0] + z, Y = chk.off[1] + y, X = chk.off[2] + x;
              float v = fnan;
              if (Z < dims[0] && Y < dims[1] && X < dims[2]) {
                const int32_t cc = col[(Z * dims[1] + Y) * dims[2] + X];
                if (cc >= 0) {
                  v = row[cc];
                  any = true;
                }
              }
              o[(z * cdim[1] + y) * cdim[2] + x] = v;
            }
        if (!any) return true;  // not stored: reads as the fill value
        return encode_chunk(c, 4, raw, chk);
      });
      for (int r = r0; ok && r < r1; ++r) {
        const char* nm = fr_feature_name((int32_t)ids[r]);
        const uint64_t h = write_chunked(w, kF32, dims, cdim, rc[r - r0], c, &fnan,
                                         {attr_i64("feature_id", {ids[r]})});
        maps_links.push_back({nm ? nm : "feature", h, false, 0, 0});
      }
    }
    GroupAddr g;
    ok = ok && write_group(w, maps_links,
                           {attr_str("layout", "dense [nz][ny][nx] float32, NaN outside the VOI")},
                           &g);
    if (ok) root.push_back({"maps", g.header, true, g.btree, g.heap});
    GroupAddr ra;
    ok = ok && write_group(w, root, root_attrs(p, src, "spatial", ids), &ra);
    ok = ok && w.finish(ra.header, ra.btree, ra.heap);
  } catch (...) {
    ok = false;
  }
  if (std::fclose(f) != 0) ok = false;
  return ok ? FR_OK : FR_ERR_IO;
}

fr_status fr_h5_write_scalar(const char* path, const fr_map_params* p, const fr_h5_source* src,
                             const double* values, int32_t n_values, const fr_h5_options* opt) {
  Codec c;
  if (!check_common(path, p, src, opt, &c) || !values) return FR_ERR_INVALID_ARG;
  const std::vector<int64_t> ids = selected_ids(p, FR_NUM_SCALAR_FEATURES);
  if ((int32_t)ids.size() != n_values || n_values < 1) return FR_ERR_INVALID_ARG;
  if (c.codec == FR_H5_GZIP && !zlib().ok) return FR_ERR_UNSUPPORTED;
  const uint64_t dims[3] = {(uint64_t)p->nz, (uint64_t)p->ny, (uint64_t)p->nx};
  uint64_t cdim[3], ng[3];
  chunk_grid(opt ? opt->chunk : kAutoChunk, dims, cdim, ng);
  FILE* f = std::fopen(path, "wb");
  if (!f) return FR_ERR_IO;
  Writer w(f);
  bool ok = true;
  try {
    std::vector<Link> root;
    std::vector<Chunk> ch;
    const int16_t fi = 0;
    const uint8_t fu = 0;
    ok = ok && volume_chunks(src->image, dims, cdim, ng, c, ch);
    if (ok)
      root.push_back({"image", write_chunked(w, kI16, dims, cdim, ch, c, &fi,
                                             {attr_str("unit", "stored intensity")}),
                      false, 0, 0});
    ok = ok && volume_chunks(src->mask, dims, cdim, ng, c, ch);
    if (ok) root.push_back({"mask", write_chunked(w, kU8, dims, cdim, ch, c, &fu, {}), false, 0, 0});
    // ordered feature names (fixed-length strings) and float64 values
    size_t len = 1;
    for (int64_t id : ids) len = std::max(len, std::strlen(fr_feature_name((int32_t)id)) + 1);
    std::vector<char> names(len * ids.size(), 0);
    for (size_t k = 0; k < ids.size(); ++k) {
      const char* nm = fr_feature_name((int32_t)ids[k]);
      std::memcpy(names.data() + k * len, nm, std::strlen(nm));
    }
    std::vector<Link> feats;
    feats.push_back({"names", write_contiguous(w, kStr, len, {(uint64_t)ids.size()}, names.data(),
                                               names.size(), {}),
                     false, 0, 0});
    feats.push_back({"values", write_contiguous(w, kF64, 0, {(uint64_t)ids.size()}, values,
                                                ids.size() * 8, {}),
                     false, 0, 0});
    GroupAddr g;
    ok = ok && write_group(w, feats, {}, &g);
    if (ok) root.push_back({"features", g.header, true, g.btree, g.heap});
    GroupAddr ra;
    ok = ok && write_group(w, root, root_attrs(p, src, "scalar", ids), &ra);
    ok = ok && w.finish(ra.header, ra.btree, ra.heap);
  } catch (...) {
    ok = false;
  }
  if (std::fclose(f) != 0) ok = false;
  return ok ? FR_OK : FR_ERR_IO;
}

}  // extern "C"
