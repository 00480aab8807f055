// Checkpoint and resume of the time-step state: pm_state_save / pm_state_load.
//
// The BDF2 recurrence of Section 3 carries u^k and u^{k-1} from step to step, and the pressure
// increment solve is warm-started from the previous q; with p^k and the step index that is the
// whole state of the time loop. A checkpoint file is
//   - a 4096-byte ASCII header: one flat JSON object, space padded, ending in '\n';
//   - the eight fields u1, u2, u3, u1_prev, u2_prev, u3_prev, p, q as little-endian IEEE-754
//     float64 arrays of n values each, in the library's node order.
// The header carries the format version, the basin's grid and physics (checked on load against the
// operator the state belongs to), an FNV-1a 64-bit hash of the ocean column list (same mask and
// column order) and one of the payload (detects a truncated or altered file).
#include <cerrno>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "pm_internal.cuh"

namespace pm {
namespace {

constexpr size_t HEADER_BYTES = 4096;
constexpr int FORMAT_VERSION = 1;
constexpr int NFIELD = 8;
const char* const FIELD_NAMES[NFIELD] = {"u1", "u2", "u3", "u1_prev", "u2_prev", "u3_prev", "p", "q"};
constexpr uint64_t FNV_OFFSET = 14695981039346656037ull;
constexpr uint64_t FNV_PRIME = 1099511628211ull;

uint64_t fnv1a(uint64_t h, const void* data, size_t bytes) {
  const unsigned char* p = static_cast<const unsigned char*>(data);
  for (size_t i = 0; i < bytes; ++i) {
    h ^= p[i];
    h *= FNV_PRIME;
  }
  return h;
}

bool host_is_little_endian() {
  const uint16_t v = 1;
  unsigned char c = 0;
  std::memcpy(&c, &v, 1);
  return c == 1;
}

uint64_t columns_hash(const pm_operator* op) {
  uint64_t h = FNV_OFFSET;
  h = fnv1a(h, op->col_i.data(), op->col_i.size() * sizeof(int32_t));
  return fnv1a(h, op->col_j.data(), op->col_j.size() * sizeof(int32_t));
}

std::string num(double v) {
  char b[40];
  std::snprintf(b, sizeof b, "%.17g", v);
  return b;
}

std::string hex64(uint64_t v) {
  char b[24];
  std::snprintf(b, sizeof b, "\"0x%016llx\"", (unsigned long long)v);
  return b;
}

// The header text for this operator and step, without the payload hash value filled in yet.
std::string header_json(const pm_operator* op, int32_t step, uint64_t payload_hash) {
  std::string js = "{\"format\":\"pm_state\",\"version\":" + std::to_string(FORMAT_VERSION) +
                   ",\"byte_order\":\"little\",\"dtype\":\"float64\"";
  js += ",\"n\":" + std::to_string(op->n) + ",\"nx\":" + std::to_string(op->nx) + ",\"ny\":" + std::to_string(op->ny) +
        ",\"nz\":" + std::to_string(op->nz) + ",\"ncols\":" + std::to_string(op->ncols);
  js += ",\"dx\":" + num(op->dx) + ",\"dy\":" + num(op->dy) + ",\"dt\":" + num(op->dt);
  js += ",\"nu\":[" + num(op->nu[0]) + "," + num(op->nu[1]) + "," + num(op->nu[2]) + "]";
  js += ",\"step\":" + std::to_string(step);
  js += ",\"fields\":[";
  for (int f = 0; f < NFIELD; ++f) js += std::string(f ? "," : "") + "\"" + FIELD_NAMES[f] + "\"";
  js += "],\"columns_fnv1a64\":" + hex64(columns_hash(op)) + ",\"payload_fnv1a64\":" + hex64(payload_hash) + "}";
  return js;
}

// Raw text of a top-level key's value in the flat header this file writes.
bool json_value(const std::string& js, const char* key, std::string* out) {
  const std::string k = std::string("\"") + key + "\":";
  size_t p = js.find(k);
  if (p == std::string::npos) return false;
  p += k.size();
  size_t e = p;
  int depth = 0;
  for (; e < js.size(); ++e) {
    const char c = js[e];
    if (c == '[') ++depth;
    else if (c == ']') --depth;
    else if ((c == ',' || c == '}') && depth == 0) break;
  }
  *out = js.substr(p, e - p);
  return true;
}

double* field_ptr(const pm_state* st, int f) {
  return f < 3 ? st->u[f] : f < 6 ? st->u_prev[f - 3] : f == 6 ? st->p : st->q;
}

int io_error(const std::string& what, const std::string& path) {
  return set_error(PM_EINVAL, what + " '" + path + "': " + std::strerror(errno));
}

}  // namespace
}  // namespace pm

extern "C" int pm_state_save(const pm_state* st, const char* path, pm_stream stream) {
  using namespace pm;
  if (!st || !path) return set_error(PM_EINVAL, "null argument");
  if (!host_is_little_endian()) return set_error(PM_EINVAL, "checkpoint files are little-endian; this host is not");
  NvtxRange range("pm_state_save");
  const pm_operator* op = st->op;
  cudaStream_t s = (cudaStream_t)stream;
  const std::string target(path);
  const std::string tmp = target + ".tmp";
  FILE* fh = std::fopen(tmp.c_str(), "wb");
  if (!fh) return io_error("cannot create", tmp);
  std::vector<char> head(HEADER_BYTES, ' ');
  std::vector<double> buf((size_t)op->n);
  uint64_t h = FNV_OFFSET;
  int st_code = PM_OK;
  if (std::fwrite(head.data(), 1, HEADER_BYTES, fh) != HEADER_BYTES) st_code = io_error("cannot write", tmp);
  for (int f = 0; f < NFIELD && st_code == PM_OK; ++f) {
    st_code = cuda_check(cudaMemcpyAsync(buf.data(), field_ptr(st, f), op->n * sizeof(double), cudaMemcpyDeviceToHost, s),
                         "checkpoint read-back");
    if (!st_code) st_code = cuda_check(cudaStreamSynchronize(s), "checkpoint read-back");
    if (st_code) break;
    h = fnv1a(h, buf.data(), buf.size() * sizeof(double));
    if (std::fwrite(buf.data(), sizeof(double), buf.size(), fh) != buf.size()) st_code = io_error("cannot write", tmp);
  }
  if (st_code == PM_OK) {
    const std::string js = header_json(op, st->step, h);
    if (js.size() + 1 > HEADER_BYTES) {
      st_code = set_error(PM_EINVAL, "checkpoint header does not fit its block");
    } else {
      std::memcpy(head.data(), js.data(), js.size());
      head[HEADER_BYTES - 1] = '\n';
      if (std::fseek(fh, 0, SEEK_SET) != 0 || std::fwrite(head.data(), 1, HEADER_BYTES, fh) != HEADER_BYTES)
        st_code = io_error("cannot write", tmp);
    }
  }
  if (std::fclose(fh) != 0 && st_code == PM_OK) st_code = io_error("cannot close", tmp);
  if (st_code == PM_OK && std::rename(tmp.c_str(), target.c_str()) != 0) st_code = io_error("cannot rename to", target);
  if (st_code != PM_OK) std::remove(tmp.c_str());
  return st_code;
}

extern "C" int pm_state_load(pm_state* st, const char* path, pm_stream stream) {
  using namespace pm;
  if (!st || !path) return set_error(PM_EINVAL, "null argument");
  if (!host_is_little_endian()) return set_error(PM_EINVAL, "checkpoint files are little-endian; this host is not");
  NvtxRange range("pm_state_load");
  const pm_operator* op = st->op;
  cudaStream_t s = (cudaStream_t)stream;
  FILE* fh = std::fopen(path, "rb");
  if (!fh) return io_error("cannot open", path);
  std::vector<char> head(HEADER_BYTES + 1, '\0');
  if (std::fread(head.data(), 1, HEADER_BYTES, fh) != HEADER_BYTES) {
    std::fclose(fh);
    return set_error(PM_EINVAL, std::string("checkpoint '") + path + "' is shorter than its header");
  }
  const std::string js(head.data());
  auto bad = [&](const std::string& why) {
    std::fclose(fh);
    return set_error(PM_EINVAL, std::string("checkpoint '") + path + "': " + why);
  };
  std::string v;
  if (!json_value(js, "format", &v) || v != "\"pm_state\"") return bad("not a pm_state checkpoint");
  if (!json_value(js, "version", &v) || v != std::to_string(FORMAT_VERSION)) return bad("unsupported version " + v);
  if (!json_value(js, "byte_order", &v) || v != "\"little\"") return bad("byte order is not little-endian");
  // the basin must be the one the state belongs to
  const char* keys[] = {"n", "nx", "ny", "nz", "ncols", "dx", "dy", "dt", "nu", "columns_fnv1a64"};
  const std::string mine = header_json(op, 0, 0);
  for (const char* k : keys) {
    std::string want;
    json_value(mine, k, &want);
    if (!json_value(js, k, &v) || v != want) return bad(std::string("saved for another basin (") + k + " " + v + ", expected " + want + ")");
  }
  if (!json_value(js, "step", &v)) return bad("no step index");
  char* end = nullptr;
  const long step = std::strtol(v.c_str(), &end, 10);
  if (end == v.c_str() || step < 0 || step > 0x7fffffffL) return bad("bad step index " + v);
  if (!json_value(js, "payload_fnv1a64", &v)) return bad("no payload hash");
  const uint64_t want_hash = std::strtoull(v.c_str() + 1, nullptr, 16);
  std::vector<double> all((size_t)NFIELD * op->n);
  const size_t got = std::fread(all.data(), sizeof(double), all.size(), fh);
  char extra = 0;
  const bool trailing = std::fread(&extra, 1, 1, fh) == 1;
  std::fclose(fh);
  if (got != all.size() || trailing) return set_error(PM_EINVAL, std::string("checkpoint '") + path + "' has the wrong payload size");
  if (fnv1a(FNV_OFFSET, all.data(), all.size() * sizeof(double)) != want_hash)
    return set_error(PM_EINVAL, std::string("checkpoint '") + path + "' payload hash mismatch (truncated or altered)");
  for (int f = 0; f < NFIELD; ++f) {
    int r = cuda_check(cudaMemcpyAsync(field_ptr(st, f), all.data() + (size_t)f * op->n, op->n * sizeof(double),
                                       cudaMemcpyHostToDevice, s), "checkpoint upload");
    if (r) return r;
  }
  // the last step's intermediate fields do not belong to the loaded state
  double* inter[] = {st->ut[0], st->ut[1], st->ut[2], st->b[0], st->b[1], st->b[2], st->bp};
  for (double* p : inter) {
    int r = cuda_check(cudaMemsetAsync(p, 0, op->n * sizeof(double), s), "checkpoint clear");
    if (r) return r;
  }
  int r = cuda_check(cudaStreamSynchronize(s), "checkpoint upload");
  if (r) return r;
  st->step = (int32_t)step;
  return PM_OK;
}
