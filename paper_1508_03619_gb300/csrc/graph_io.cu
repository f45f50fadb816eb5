// graph_io.cu — reading graphs from files and serializing built graphs (paper
// §3: the reference infrastructure loads METIS, Matrix Market and a plain-text
// edge list, and can serialize a built graph so that later runs skip the build).
//
// Text formats are parsed on the host into an edge list (src[i] -> dst[i]),
// which the device builder turns into a graph like any other edge list.  The
// serialized format stores the in-direction CSR exactly as the handle holds it,
// so loading it copies two arrays to the device and re-derives only the
// out-degrees and degree statistics (after a structure check on the device).
//
// Serialized file (little-endian, 64-byte header):
//   0  char[8]  magic "GAPCSC\0\1"
//   8  u32      format version (1)
//  12  u32      header bytes (64)
//  16  i64      n (vertices)
//  24  i64      m (stored arcs)
//  32  u32      construction flags (GAP_SYMMETRIZE | GAP_DEDUP | GAP_DROP_SELF_LOOPS)
//  36  u32      byte-order tag 0x01020304
//  40  u64      payload checksum (below)
//  48  16 bytes zero
//  64  i64[n+1] in_off, then i32[m] in_idx
// Checksum: the payload read as 64-bit little-endian words w_i (the last word
// zero-padded), sum over i of mix(w_i + (i+1) * 0x9E3779B97F4A7C15) modulo 2^64,
// with mix the splitmix64 finalizer (Steele, Lea & Flood 2014): order-sensitive
// through the index, and computable in any order.
#include <ctype.h>
#include <errno.h>
#include <stdlib.h>
#include <string.h>
#include <strings.h>

#include <new>
#include <vector>

#include "graph.cuh"

struct gap_edge_list {
  int64_t n = 0;
  uint32_t implied_flags = 0;
  int32_t format = 0;
  std::vector<int32_t> src, dst;
};

namespace gap {
namespace {

constexpr int64_t kMaxId = 2147483646;  // ids in [0, 2^31 - 2] so that n <= 2^31 - 1
constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;
constexpr uint32_t kVersion = 1;
constexpr uint32_t kOrderTag = 0x01020304u;
const char kMagic[8] = {'G', 'A', 'P', 'C', 'S', 'C', '\0', '\1'};
constexpr size_t kStage = size_t(64) << 20;  // host staging chunk for the serialized arrays

struct FileHeader {
  char magic[8];
  uint32_t version;
  uint32_t header_bytes;
  int64_t n;
  int64_t m;
  uint32_t flags;
  uint32_t order_tag;
  uint64_t checksum;
  uint8_t pad[16];
};
static_assert(sizeof(FileHeader) == 64, "header is 64 bytes");

inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Running payload checksum over a byte stream fed in pieces of any size.
struct Checksum {
  uint64_t sum = 0;
  uint64_t word_index = 0;
  uint8_t part[8];
  int npart = 0;
  void add_word(uint64_t w) { sum += mix64(w + (++word_index) * kGolden); }
  void feed(const void* p, size_t bytes) {
    const uint8_t* b = static_cast<const uint8_t*>(p);
    while (bytes > 0 && npart > 0) {
      part[npart++] = *b++;
      --bytes;
      if (npart == 8) {
        uint64_t w;
        memcpy(&w, part, 8);
        add_word(w);
        npart = 0;
      }
    }
    while (bytes >= 8) {
      uint64_t w;
      memcpy(&w, b, 8);
      add_word(w);
      b += 8;
      bytes -= 8;
    }
    while (bytes > 0) {
      part[npart++] = *b++;
      --bytes;
    }
  }
  uint64_t finish() {
    if (npart > 0) {
      memset(part + npart, 0, 8 - npart);
      uint64_t w;
      memcpy(&w, part, 8);
      add_word(w);
      npart = 0;
    }
    return sum;
  }
};

// Buffered line reader; a line may span buffer refills.
class LineReader {
 public:
  explicit LineReader(FILE* f) : f_(f), buf_(size_t(16) << 20) {}
  // Next line without its terminator ('\n', "\r\n"); false at end of file.
  bool next(const char** b, const char** e) {
    for (;;) {
      const char* p = static_cast<const char*>(memchr(buf_.data() + pos_, '\n', len_ - pos_));
      if (p) {
        *b = buf_.data() + pos_;
        *e = p;
        pos_ = (size_t)(p - buf_.data()) + 1;
        trim_cr(*b, e);
        ++line_;
        return true;
      }
      if (eof_) {
        if (pos_ < len_) {
          *b = buf_.data() + pos_;
          *e = buf_.data() + len_;
          pos_ = len_;
          trim_cr(*b, e);
          ++line_;
          return true;
        }
        return false;
      }
      refill();
    }
  }
  int64_t line() const { return line_; }
  bool read_error() const { return ferror(f_) != 0; }

 private:
  static void trim_cr(const char* b, const char** e) {
    if (*e > b && (*e)[-1] == '\r') --*e;
  }
  void refill() {
    if (pos_ > 0) {
      memmove(buf_.data(), buf_.data() + pos_, len_ - pos_);
      len_ -= pos_;
      pos_ = 0;
    }
    if (len_ == buf_.size()) buf_.resize(buf_.size() * 2);  // a line longer than the buffer
    const size_t got = fread(buf_.data() + len_, 1, buf_.size() - len_, f_);
    len_ += got;
    if (got == 0) eof_ = true;
  }
  FILE* f_;
  std::vector<char> buf_;
  size_t pos_ = 0, len_ = 0;
  bool eof_ = false;
  int64_t line_ = 0;
};

inline const char* skip_space(const char* p, const char* e) {
  while (p < e && (*p == ' ' || *p == '\t' || *p == '\v' || *p == '\f')) ++p;
  return p;
}

// Decimal integer token at *p (optional sign); advances *p past it.  Returns
// false if there is no token; *bad set if the token is not an integer.
bool int_token(const char** p, const char* e, int64_t* v, bool* bad) {
  const char* q = skip_space(*p, e);
  if (q == e) return false;
  bool neg = false;
  if (*q == '+' || *q == '-') {
    neg = *q == '-';
    ++q;
  }
  if (q == e || !isdigit((unsigned char)*q)) {
    *bad = true;
    return false;
  }
  int64_t x = 0;
  while (q < e && isdigit((unsigned char)*q)) {
    if (x > (INT64_MAX - 9) / 10) {
      *bad = true;
      return false;
    }
    x = x * 10 + (*q - '0');
    ++q;
  }
  if (q < e && !(*q == ' ' || *q == '\t' || *q == '\v' || *q == '\f')) {
    *bad = true;  // e.g. "12x" or a real number where an id belongs
    return false;
  }
  *v = neg ? -x : x;
  *p = q;
  return true;
}

bool blank(const char* b, const char* e) { return skip_space(b, e) == e; }

// Next whitespace-separated word (for headers).
bool word(const char** p, const char* e, std::string* w) {
  const char* q = skip_space(*p, e);
  if (q == e) return false;
  const char* s = q;
  while (q < e && !(*q == ' ' || *q == '\t' || *q == '\v' || *q == '\f')) ++q;
  w->assign(s, q);
  *p = q;
  return true;
}

gap_status parse_error(const char* path, int64_t line, const char* what) {
  set_error("%s:%lld: %s", path, (long long)line, what);
  return GAP_ERR_INVALID_ARG;
}

gap_status push_arc(gap_edge_list* el, int64_t u, int64_t v) {
  try {
    el->src.push_back((int32_t)u);
    el->dst.push_back((int32_t)v);
  } catch (...) {
    set_error("out of host memory after %zu arcs", el->src.size());
    return GAP_ERR_OOM;
  }
  return GAP_OK;
}

// Plain text: one arc "u v" per line, 0-based ids; further columns (a weight)
// are ignored; lines starting with '#' or '%' and blank lines are skipped.
// n = 1 + the largest id.
gap_status read_edge_list(FILE* f, const char* path, gap_edge_list* el) {
  LineReader r(f);
  const char *b, *e;
  int64_t maxid = -1;
  while (r.next(&b, &e)) {
    const char* p = skip_space(b, e);
    if (p == e || *p == '#' || *p == '%') continue;
    int64_t u, v;
    bool bad = false;
    if (!int_token(&p, e, &u, &bad) || !int_token(&p, e, &v, &bad))
      return parse_error(path, r.line(), "expected two integer vertex ids");
    if (u < 0 || v < 0 || u > kMaxId || v > kMaxId)
      return parse_error(path, r.line(), "vertex id outside [0, 2^31 - 2]");
    maxid = u > maxid ? u : maxid;
    maxid = v > maxid ? v : maxid;
    GAP_TRY(push_arc(el, u, v));
  }
  if (r.read_error()) return parse_error(path, r.line(), "read error");
  el->n = maxid + 1;
  return GAP_OK;
}

// Matrix Market coordinate format: entry (i, j) is the arc i-1 -> j-1; values
// are ignored.  A symmetric, skew-symmetric or Hermitian matrix stores one
// triangle, so the graph it names is the symmetrized one (GAP_SYMMETRIZE is
// implied).  n = max(rows, cols).
gap_status read_matrix_market(FILE* f, const char* path, gap_edge_list* el) {
  LineReader r(f);
  const char *b, *e;
  if (!r.next(&b, &e)) return parse_error(path, 1, "empty file");
  std::string banner, object, format, field, symmetry;
  const char* p = b;
  if (!word(&p, e, &banner) || strcasecmp(banner.c_str(), "%%MatrixMarket") != 0 || !word(&p, e, &object) ||
      !word(&p, e, &format) || !word(&p, e, &field) || !word(&p, e, &symmetry))
    return parse_error(path, 1, "expected '%%MatrixMarket matrix coordinate <field> <symmetry>'");
  if (strcasecmp(object.c_str(), "matrix") != 0) return parse_error(path, 1, "object is not 'matrix'");
  if (strcasecmp(format.c_str(), "coordinate") != 0)
    return parse_error(path, 1, "only the 'coordinate' (sparse) format names a graph");
  const char* fields[] = {"pattern", "real", "integer", "double", "complex"};
  bool field_ok = false;
  for (const char* fl : fields) field_ok |= strcasecmp(field.c_str(), fl) == 0;
  if (!field_ok) return parse_error(path, 1, "unknown field (pattern, real, integer, double, complex)");
  if (strcasecmp(symmetry.c_str(), "general") == 0) {
    el->implied_flags = 0;
  } else if (strcasecmp(symmetry.c_str(), "symmetric") == 0 || strcasecmp(symmetry.c_str(), "skew-symmetric") == 0 ||
             strcasecmp(symmetry.c_str(), "hermitian") == 0) {
    el->implied_flags = GAP_SYMMETRIZE;
  } else {
    return parse_error(path, 1, "unknown symmetry (general, symmetric, skew-symmetric, hermitian)");
  }
  int64_t rows = -1, cols = -1, nnz = -1;
  while (r.next(&b, &e)) {
    p = skip_space(b, e);
    if (p == e || *p == '%') continue;
    bool bad = false;
    if (!int_token(&p, e, &rows, &bad) || !int_token(&p, e, &cols, &bad) || !int_token(&p, e, &nnz, &bad) ||
        !blank(p, e))
      return parse_error(path, r.line(), "expected the size line 'rows cols entries'");
    break;
  }
  if (nnz < 0 || rows < 0 || cols < 0) return parse_error(path, r.line(), "missing or negative size line");
  if (rows > kMaxId + 1 || cols > kMaxId + 1) return parse_error(path, r.line(), "more than 2^31 - 1 vertices");
  try {
    el->src.reserve((size_t)nnz);
    el->dst.reserve((size_t)nnz);
  } catch (...) {
    set_error("out of host memory for %lld entries", (long long)nnz);
    return GAP_ERR_OOM;
  }
  int64_t seen = 0;
  while (r.next(&b, &e)) {
    p = skip_space(b, e);
    if (p == e || *p == '%') continue;
    int64_t i, j;
    bool bad = false;
    if (!int_token(&p, e, &i, &bad) || !int_token(&p, e, &j, &bad))
      return parse_error(path, r.line(), "expected an entry 'row col [value]'");
    if (i < 1 || i > rows || j < 1 || j > cols) return parse_error(path, r.line(), "entry outside the matrix");
    if (++seen > nnz) return parse_error(path, r.line(), "more entries than the size line states");
    GAP_TRY(push_arc(el, i - 1, j - 1));
  }
  if (r.read_error()) return parse_error(path, r.line(), "read error");
  if (seen < nnz) return parse_error(path, r.line(), "fewer entries than the size line states");
  el->n = rows > cols ? rows : cols;
  return GAP_OK;
}

// METIS graph format: header "n m [fmt [ncon]]"; then one line per vertex i
// (1-based) listing its neighbours, each an arc i-1 -> j-1.  fmt's last digit
// says each neighbour is followed by an edge weight, its middle digit that the
// line starts with ncon vertex weights, its first digit that it starts with a
// vertex size; all weights are skipped.  Lines starting with '%' are comments;
// a blank line is a vertex without neighbours.  METIS lists every undirected
// edge from both ends, so the arcs read must number 2m.
gap_status read_metis(FILE* f, const char* path, gap_edge_list* el) {
  LineReader r(f);
  const char *b, *e;
  int64_t n = -1, m = -1, fmt = 0, ncon = 0;
  while (r.next(&b, &e)) {
    const char* p = skip_space(b, e);
    if (p == e || *p == '%') continue;
    bool bad = false;
    if (!int_token(&p, e, &n, &bad) || !int_token(&p, e, &m, &bad))
      return parse_error(path, r.line(), "expected the header 'n m [fmt [ncon]]'");
    if (int_token(&p, e, &fmt, &bad)) {
      if (!int_token(&p, e, &ncon, &bad) && bad) return parse_error(path, r.line(), "bad ncon in the header");
    } else if (bad) {
      return parse_error(path, r.line(), "bad fmt in the header");
    }
    if (!blank(p, e)) return parse_error(path, r.line(), "extra tokens in the header");
    break;
  }
  if (n < 0 || m < 0) return parse_error(path, r.line(), "missing or negative header");
  if (n > kMaxId + 1) return parse_error(path, r.line(), "more than 2^31 - 1 vertices");
  if (fmt < 0 || fmt > 111 || (fmt % 10) > 1 || ((fmt / 10) % 10) > 1 || (fmt / 100) > 1)
    return parse_error(path, r.line(), "fmt must be a 3-digit code of 0s and 1s");
  const bool ew = fmt % 10 == 1, vw = (fmt / 10) % 10 == 1, vs = fmt / 100 == 1;
  if (vw && ncon == 0) ncon = 1;
  if (!vw) ncon = 0;
  try {
    el->src.reserve((size_t)(2 * m));
    el->dst.reserve((size_t)(2 * m));
  } catch (...) {
    set_error("out of host memory for %lld edges", (long long)m);
    return GAP_ERR_OOM;
  }
  int64_t v = 0;
  while (v < n && r.next(&b, &e)) {
    const char* p = skip_space(b, e);
    if (p < e && *p == '%') continue;
    bool bad = false;
    int64_t skip;
    for (int64_t k = 0; k < (vs ? 1 : 0) + ncon; ++k)
      if (!int_token(&p, e, &skip, &bad)) return parse_error(path, r.line(), "missing vertex size or weight");
    int64_t j;
    while (int_token(&p, e, &j, &bad)) {
      if (j < 1 || j > n) return parse_error(path, r.line(), "neighbour outside [1, n]");
      GAP_TRY(push_arc(el, v, j - 1));
      if (ew && !int_token(&p, e, &skip, &bad)) return parse_error(path, r.line(), "missing edge weight");
    }
    if (bad) return parse_error(path, r.line(), "expected integer neighbour ids");
    ++v;
  }
  if (r.read_error()) return parse_error(path, r.line(), "read error");
  if (v < n) return parse_error(path, r.line(), "fewer vertex lines than n");
  while (r.next(&b, &e)) {
    const char* p = skip_space(b, e);
    if (p != e && *p != '%') return parse_error(path, r.line(), "more vertex lines than n");
  }
  if ((int64_t)el->src.size() != 2 * m)
    return parse_error(path, r.line(), "the adjacency lists hold a number of arcs other than 2m");
  el->n = n;
  return GAP_OK;
}

bool ends_with(const char* s, const char* suf) {
  const size_t a = strlen(s), b = strlen(suf);
  return a >= b && strcasecmp(s + a - b, suf) == 0;
}

int32_t format_of(const char* path, int32_t format) {
  if (format != GAP_FMT_AUTO) return format;
  if (ends_with(path, ".el") || ends_with(path, ".txt")) return GAP_FMT_EDGE_LIST;
  if (ends_with(path, ".mtx")) return GAP_FMT_MATRIX_MARKET;
  if (ends_with(path, ".graph") || ends_with(path, ".metis")) return GAP_FMT_METIS;
  if (ends_with(path, ".gcsc")) return GAP_FMT_SERIALIZED;
  return -1;
}

struct FileCloser {
  FILE* f;
  ~FileCloser() {
    if (f) fclose(f);
  }
};

gap_status read_text(const char* path, int32_t format, gap_edge_list** out) {
  FILE* f = fopen(path, "rb");
  if (!f) {
    set_error("cannot open %s: %s", path, strerror(errno));
    return GAP_ERR_INVALID_ARG;
  }
  FileCloser fc{f};
  gap_edge_list* el = new (std::nothrow) gap_edge_list();
  if (!el) {
    set_error("out of host memory");
    return GAP_ERR_OOM;
  }
  el->format = format;
  gap_status st;
  if (format == GAP_FMT_EDGE_LIST) st = read_edge_list(f, path, el);
  else if (format == GAP_FMT_MATRIX_MARKET) st = read_matrix_market(f, path, el);
  else st = read_metis(f, path, el);
  if (st != GAP_OK) {
    delete el;
    return st;
  }
  *out = el;
  return GAP_OK;
}

// Pinned staging buffer for streaming the serialized arrays.
struct Pinned {
  void* p = nullptr;
  ~Pinned() {
    if (p) cudaFreeHost(p);
  }
};

gap_status read_header(FILE* f, const char* path, FileHeader* h) {
  if (fread(h, 1, sizeof(*h), f) != sizeof(*h)) {
    set_error("%s: shorter than the 64-byte header", path);
    return GAP_ERR_INVALID_ARG;
  }
  if (memcmp(h->magic, kMagic, 8) != 0) {
    set_error("%s: not a serialized gap graph (bad magic)", path);
    return GAP_ERR_INVALID_ARG;
  }
  if (h->order_tag != kOrderTag) {
    set_error("%s: written with another byte order", path);
    return GAP_ERR_INVALID_ARG;
  }
  if (h->version != kVersion || h->header_bytes != sizeof(FileHeader)) {
    set_error("%s: unsupported version %u", path, h->version);
    return GAP_ERR_INVALID_ARG;
  }
  if (h->n < 1 || h->n > kMaxId + 1 || h->m < 0 || h->m > (int64_t(1) << 40)) {
    set_error("%s: n = %lld or m = %lld out of range", path, (long long)h->n, (long long)h->m);
    return GAP_ERR_INVALID_ARG;
  }
  if (fseeko(f, 0, SEEK_END) != 0) {
    set_error("%s: cannot seek", path);
    return GAP_ERR_INVALID_ARG;
  }
  const int64_t size = (int64_t)ftello(f);
  const int64_t want = (int64_t)sizeof(FileHeader) + 8 * (h->n + 1) + 4 * h->m;
  if (size != want) {
    set_error("%s: %lld bytes, the header implies %lld", path, (long long)size, (long long)want);
    return GAP_ERR_INVALID_ARG;
  }
  if (fseeko(f, (off_t)sizeof(FileHeader), SEEK_SET) != 0) {
    set_error("%s: cannot seek", path);
    return GAP_ERR_INVALID_ARG;
  }
  return GAP_OK;
}

// Stream `bytes` from the file into device memory `dst` through the pinned
// staging buffer, feeding the checksum.
gap_status file_to_device(FILE* f, const char* path, void* dst, size_t bytes, void* stage, cudaStream_t s,
                          Checksum* ck, int64_t* first_last /* int64 offsets: first and last word, or null */) {
  size_t done = 0;
  while (done < bytes) {
    const size_t len = bytes - done < kStage ? bytes - done : kStage;
    GAP_CUDA(cudaStreamSynchronize(s));  // the previous chunk's copy left the staging buffer
    if (fread(stage, 1, len, f) != len) {
      set_error("%s: read error", path);
      return GAP_ERR_INVALID_ARG;
    }
    ck->feed(stage, len);
    if (first_last) {
      if (done == 0) memcpy(&first_last[0], stage, 8);
      if (done + len == bytes) memcpy(&first_last[1], static_cast<char*>(stage) + len - 8, 8);
    }
    GAP_CUDA(cudaMemcpyAsync(static_cast<char*>(dst) + done, stage, len, cudaMemcpyHostToDevice, s));
    done += len;
  }
  GAP_CUDA(cudaStreamSynchronize(s));
  return GAP_OK;
}

gap_status device_to_file(FILE* f, const char* path, const void* src, size_t bytes, void* stage, cudaStream_t s,
                          Checksum* ck) {
  size_t done = 0;
  while (done < bytes) {
    const size_t len = bytes - done < kStage ? bytes - done : kStage;
    GAP_CUDA(cudaMemcpyAsync(stage, static_cast<const char*>(src) + done, len, cudaMemcpyDeviceToHost, s));
    GAP_CUDA(cudaStreamSynchronize(s));
    if (ck) ck->feed(stage, len);
    if (f && fwrite(stage, 1, len, f) != len) {
      set_error("%s: write error: %s", path, strerror(errno));
      return GAP_ERR_INVALID_ARG;
    }
    done += len;
  }
  return GAP_OK;
}

gap_status load_serialized(const char* path, cudaStream_t s, gap_graph** out) {
  FILE* f = fopen(path, "rb");
  if (!f) {
    set_error("cannot open %s: %s", path, strerror(errno));
    return GAP_ERR_INVALID_ARG;
  }
  FileCloser fc{f};
  FileHeader h;
  GAP_TRY(read_header(f, path, &h));
  const int64_t n = h.n, m = h.m;
  Pinned stage;
  if (cudaMallocHost(&stage.p, kStage) != cudaSuccess) {
    cudaGetLastError();
    set_error("pinned staging allocation failed");
    return GAP_ERR_OOM;
  }
  int64_t* d_off = nullptr;
  int32_t* d_idx = nullptr;
  if (cudaMalloc(&d_off, sizeof(int64_t) * (n + 1)) != cudaSuccess ||
      cudaMalloc(&d_idx, sizeof(int32_t) * (m > 0 ? m : 1)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(d_off);
    set_error("graph allocation failed");
    return GAP_ERR_OOM;
  }
  Checksum ck;
  int64_t ends[2] = {0, 0};
  gap_status st = file_to_device(f, path, d_off, sizeof(int64_t) * (n + 1), stage.p, s, &ck, ends);
  if (st == GAP_OK) st = file_to_device(f, path, d_idx, sizeof(int32_t) * m, stage.p, s, &ck, nullptr);
  if (st == GAP_OK && ck.finish() != h.checksum) {
    set_error("%s: checksum mismatch (file damaged)", path);
    st = GAP_ERR_INVALID_ARG;
  }
  if (st == GAP_OK && (ends[0] != 0 || ends[1] != m)) {
    set_error("%s: offsets must start at 0 and end at m", path);
    st = GAP_ERR_INVALID_ARG;
  }
  if (st != GAP_OK) {
    cudaStreamSynchronize(s);
    cudaFree(d_off);
    cudaFree(d_idx);
    return st;
  }
  return graph_from_csc(n, m, d_off, d_idx, h.flags, s, out);
}

}  // namespace
}  // namespace gap

using namespace gap;

extern "C" {

gap_status gap_edge_list_read(const char* path, int32_t format, gap_edge_list_t** out) {
  clear_error();
  if (!path || !out) {
    set_error("path or out is NULL");
    return GAP_ERR_INVALID_ARG;
  }
  *out = nullptr;
  const int32_t fmt = format_of(path, format);
  if (fmt != GAP_FMT_EDGE_LIST && fmt != GAP_FMT_MATRIX_MARKET && fmt != GAP_FMT_METIS) {
    set_error("%s: not a text graph format (give GAP_FMT_EDGE_LIST, _MATRIX_MARKET or _METIS, or a "
              ".el/.txt/.mtx/.graph/.metis suffix)", path);
    return GAP_ERR_INVALID_ARG;
  }
  return read_text(path, fmt, out);
}

gap_status gap_edge_list_info(const gap_edge_list_t* e, int64_t* n, int64_t* m, uint32_t* implied_flags) {
  clear_error();
  if (!e) {
    set_error("edge list is NULL");
    return GAP_ERR_INVALID_ARG;
  }
  if (n) *n = e->n;
  if (m) *m = (int64_t)e->src.size();
  if (implied_flags) *implied_flags = e->implied_flags;
  return GAP_OK;
}

gap_status gap_edge_list_arrays(const gap_edge_list_t* e, const int32_t** src, const int32_t** dst) {
  clear_error();
  if (!e || !src || !dst) {
    set_error("NULL argument");
    return GAP_ERR_INVALID_ARG;
  }
  *src = e->src.data();
  *dst = e->dst.data();
  return GAP_OK;
}

void gap_edge_list_destroy(gap_edge_list_t* e) { delete e; }

gap_status gap_graph_load(const char* path, int32_t format, uint32_t flags, void* stream, gap_graph_t** out) {
  NvtxRange nv_call("gap_graph_load");
  clear_error();
  if (!path || !out) {
    set_error("path or out is NULL");
    return GAP_ERR_INVALID_ARG;
  }
  *out = nullptr;
  const int32_t fmt = format_of(path, format);
  cudaStream_t s = (cudaStream_t)stream;
  if (fmt == GAP_FMT_SERIALIZED) return load_serialized(path, s, out);
  if (fmt != GAP_FMT_EDGE_LIST && fmt != GAP_FMT_MATRIX_MARKET && fmt != GAP_FMT_METIS) {
    set_error("%s: unknown graph format %d (no known suffix)", path, (int)format);
    return GAP_ERR_INVALID_ARG;
  }
  if (flags & GAP_INPUT_ON_DEVICE) {
    set_error("GAP_INPUT_ON_DEVICE does not apply to files");
    return GAP_ERR_INVALID_ARG;
  }
  gap_edge_list* el = nullptr;
  GAP_TRY(read_text(path, fmt, &el));
  if (el->n < 1) {
    delete el;
    set_error("%s: the file names no vertex", path);
    return GAP_ERR_INVALID_ARG;
  }
  const gap_status st = gap_graph_create_from_edges(el->n, (int64_t)el->src.size(), el->src.data(), el->dst.data(),
                                                    flags | el->implied_flags, stream, out);
  delete el;
  return st;
}

gap_status gap_graph_save(gap_graph_t* g, const char* path, void* stream) {
  NvtxRange nv_call("gap_graph_save");
  clear_error();
  if (!g || !path) {
    set_error("graph or path is NULL");
    return GAP_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (g->has_run) GAP_CUDA(cudaStreamSynchronize(g->last_stream));
  Pinned stage;
  if (cudaMallocHost(&stage.p, kStage) != cudaSuccess) {
    cudaGetLastError();
    set_error("pinned staging allocation failed");
    return GAP_ERR_OOM;
  }
  // the checksum goes into the header, so the arrays are read twice: once to
  // sum them, once to write them
  Checksum ck;
  GAP_TRY(device_to_file(nullptr, path, g->in_off, sizeof(int64_t) * (g->n + 1), stage.p, s, &ck));
  GAP_TRY(device_to_file(nullptr, path, g->in_idx, sizeof(int32_t) * g->m, stage.p, s, &ck));
  FileHeader h;
  memset(&h, 0, sizeof(h));
  memcpy(h.magic, kMagic, 8);
  h.version = kVersion;
  h.header_bytes = sizeof(FileHeader);
  h.n = g->n;
  h.m = g->m;
  h.flags = g->build_flags;
  h.order_tag = kOrderTag;
  h.checksum = ck.finish();
  FILE* f = fopen(path, "wb");
  if (!f) {
    set_error("cannot create %s: %s", path, strerror(errno));
    return GAP_ERR_INVALID_ARG;
  }
  gap_status st = GAP_OK;
  if (fwrite(&h, 1, sizeof(h), f) != sizeof(h)) {
    set_error("%s: write error: %s", path, strerror(errno));
    st = GAP_ERR_INVALID_ARG;
  }
  if (st == GAP_OK) st = device_to_file(f, path, g->in_off, sizeof(int64_t) * (g->n + 1), stage.p, s, nullptr);
  if (st == GAP_OK) st = device_to_file(f, path, g->in_idx, sizeof(int32_t) * g->m, stage.p, s, nullptr);
  if (fclose(f) != 0 && st == GAP_OK) {
    set_error("%s: close failed: %s", path, strerror(errno));
    st = GAP_ERR_INVALID_ARG;
  }
  if (st != GAP_OK) remove(path);
  return st;
}

gap_status gap_graph_build_flags(const gap_graph_t* g, uint32_t* flags) {
  clear_error();
  if (!g || !flags) {
    set_error("NULL argument");
    return GAP_ERR_INVALID_ARG;
  }
  *flags = g->build_flags;
  return GAP_OK;
}

}  // extern "C"
