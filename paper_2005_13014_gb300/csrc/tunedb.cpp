// tunedb.cpp - the tuning database: the best schedule the autotuner found
// for a (program, dtype, domain extent, field strides, alignment, device)
// key, with its time, kept in memory and in a text file. The paper tunes
// unroll factors empirically (§VII-C); the database keeps the results across
// runs, so a later autotune of the same case takes the recorded schedule
// without timing anything.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/oec.h"
#include "api_internal.h"

using namespace oec;

struct oec_tunedb {
  std::string path;
  struct Entry {
    oec_schedule s;
    double ms;
  };
  std::map<std::string, Entry> entries;
  std::mutex mu;
};

namespace {

const char* kHeader = "oec-tunedb 1";

uint64_t fnv1a64(const std::string& t) {
  uint64_t h = 1469598103934665603ull;
  for (unsigned char c : t) {
    h ^= c;
    h *= 1099511628211ull;
  }
  return h;
}

// the key of an apply: program (canonical text, kind, dtype), domain extent,
// shared j/k strides, whether every field's domain corner and the strides are
// 16-byte aligned (the vector and TMA schedules need it) and the device
int make_key(const oec_program* p, const oec_field_desc* in, int n_in, const oec_field_desc* out, int n_out,
             const int64_t lb[3], const int64_t ub[3], std::string& key) {
  if (!p || !lb || !ub || (n_in && !in) || n_out < 1 || !out) return fail(OEC_ERR_INVALID_ARG, "null argument");
  if (n_in != (int)p->ir.inputs.size() || n_out != (int)p->ir.outputs.size())
    return fail(OEC_ERR_INVALID_ARG, "field counts do not match the program");
  const size_t es = elem_size(p->dtype);
  const int64_t sj = out[0].stride[1], sk = out[0].stride[2];
  bool a16 = (sj * (int64_t)es) % 16 == 0 && (sk * (int64_t)es) % 16 == 0;
  for (int x = 0; x < n_in + n_out; ++x) {
    const oec_field_desc& f = x < n_in ? in[x] : out[x - n_in];
    int64_t off = 0;
    for (int d = 0; d < 3; ++d) off += (f.origin[d] + lb[d]) * f.stride[d];
    a16 = a16 && (((uintptr_t)f.data + off * (int64_t)es) % 16 == 0) && ((uintptr_t)f.data % 16 == 0);
  }
  std::string dev = "none";
  int d = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&d) == cudaSuccess && cudaGetDeviceProperties(&prop, d) == cudaSuccess) {
    std::ostringstream o;
    o << prop.name << "/" << prop.multiProcessorCount << "sm/cc" << prop.major << prop.minor;
    dev = o.str();
  } else {
    cudaGetLastError();
  }
  for (char& c : dev)
    if (c == '\t' || c == '\n' || c == '|') c = ' ';
  char h[17];
  std::snprintf(h, sizeof h, "%016llx", (unsigned long long)fnv1a64(canonical(p->ir)));
  std::ostringstream k;
  k << h << "|kind" << p->kind << "|" << (p->dtype == OEC_F64 ? "f64" : "f32") << "|" << (ub[0] - lb[0]) << "x"
    << (ub[1] - lb[1]) << "x" << (ub[2] - lb[2]) << "|sj" << sj << "|sk" << sk << "|a16=" << (a16 ? 1 : 0) << "|"
    << dev;
  key = k.str();
  return OEC_OK;
}

bool parse_line(const std::string& line, std::string& key, oec_tunedb::Entry& e) {
  const size_t t1 = line.find('\t'), t2 = t1 == std::string::npos ? t1 : line.find('\t', t1 + 1);
  if (t1 == std::string::npos || t2 == std::string::npos) return false;
  key = line.substr(0, t1);
  std::istringstream f(line.substr(t1 + 1, t2 - t1 - 1));
  e.s = oec_schedule{};
  if (!(f >> e.s.fusion >> e.s.staging >> e.s.tile_i >> e.s.tile_j >> e.s.unroll >> e.s.k_chunk >> e.s.arith))
    return false;
  if (!(f >> e.s.index_bits)) e.s.index_bits = OEC_INDEX_AUTO;   // entries written before the field existed
  if (!(f >> e.s.sweep >> e.s.slabs)) e.s.sweep = e.s.slabs = 0;   // likewise
  std::istringstream m(line.substr(t2 + 1));
  return (bool)(m >> e.ms) && !key.empty();
}

}  // namespace

int oec_tunedb_open(const char* path, oec_tunedb_t* out) {
  clear_error();
  if (!out) return fail(OEC_ERR_INVALID_ARG, "null output handle");
  *out = nullptr;
  oec_tunedb* db = new (std::nothrow) oec_tunedb();
  if (!db) return fail(OEC_ERR_INVALID_ARG, "out of host memory");
  if (path) {
    db->path = path;
    std::ifstream f(path);
    if (f) {
      std::string line;
      if (!std::getline(f, line) || line != kHeader) {
        delete db;
        return fail(OEC_ERR_INVALID_ARG, "%s: not a tuning database", path);
      }
      int n = 1;
      while (std::getline(f, line)) {
        ++n;
        if (line.empty()) continue;
        std::string key;
        oec_tunedb::Entry e;
        if (!parse_line(line, key, e)) {
          delete db;
          return fail(OEC_ERR_INVALID_ARG, "%s:%d: malformed entry", path, n);
        }
        db->entries[key] = e;
      }
    }
  }
  *out = db;
  return OEC_OK;
}

int oec_tunedb_save(oec_tunedb_t db, const char* path) {
  clear_error();
  if (!db) return fail(OEC_ERR_INVALID_ARG, "null database");
  const std::string dst = path ? std::string(path) : db->path;
  if (dst.empty()) return fail(OEC_ERR_INVALID_ARG, "database opened without a path, and none given");
  const std::string tmp = dst + ".tmp";
  {
    std::lock_guard<std::mutex> g(db->mu);
    std::ofstream f(tmp, std::ios::trunc);
    if (!f) return fail(OEC_ERR_INVALID_ARG, "%s: cannot write", tmp.c_str());
    f << kHeader << "\n";
    f.precision(9);
    for (const auto& kv : db->entries) {
      const oec_schedule& s = kv.second.s;
      f << kv.first << "\t" << s.fusion << " " << s.staging << " " << s.tile_i << " " << s.tile_j << " " << s.unroll
        << " " << s.k_chunk << " " << s.arith << " " << s.index_bits << " " << s.sweep << " " << s.slabs << "\t"
        << kv.second.ms << "\n";
    }
    if (!f) return fail(OEC_ERR_INVALID_ARG, "%s: write failed", tmp.c_str());
  }
  if (std::rename(tmp.c_str(), dst.c_str()) != 0) return fail(OEC_ERR_INVALID_ARG, "%s: cannot replace", dst.c_str());
  return OEC_OK;
}

int oec_tunedb_count(oec_tunedb_t db) {
  clear_error();
  if (!db) return fail(OEC_ERR_INVALID_ARG, "null database");
  std::lock_guard<std::mutex> g(db->mu);
  return (int)db->entries.size();
}

void oec_tunedb_close(oec_tunedb_t db) { delete db; }

int oec_tunedb_find(oec_tunedb_t db, oec_program_t p, const oec_field_desc* in, int n_in, const oec_field_desc* out,
                    int n_out, const int64_t lb[3], const int64_t ub[3], oec_schedule* s, double* ms, int* found) {
  clear_error();
  if (!db || !found) return fail(OEC_ERR_INVALID_ARG, "null argument");
  *found = 0;
  std::string key;
  const int rc = make_key(p, in, n_in, out, n_out, lb, ub, key);
  if (rc) return rc;
  std::lock_guard<std::mutex> g(db->mu);
  auto it = db->entries.find(key);
  if (it == db->entries.end()) return OEC_OK;
  *found = 1;
  if (s) *s = it->second.s;
  if (ms) *ms = it->second.ms;
  return OEC_OK;
}

int oec_tunedb_record(oec_tunedb_t db, oec_program_t p, const oec_field_desc* in, int n_in, const oec_field_desc* out,
                      int n_out, const int64_t lb[3], const int64_t ub[3], const oec_schedule* s, double ms) {
  clear_error();
  if (!db || !s) return fail(OEC_ERR_INVALID_ARG, "null argument");
  std::string why;
  if (!schedule_ok(p ? p->kind : 0, *s, why)) return fail(OEC_ERR_UNSUPPORTED, "schedule: %s", why.c_str());
  std::string key;
  const int rc = make_key(p, in, n_in, out, n_out, lb, ub, key);
  if (rc) return rc;
  std::lock_guard<std::mutex> g(db->mu);
  db->entries[key] = oec_tunedb::Entry{*s, ms};
  return OEC_OK;
}

int oec_program_autotune_db(oec_program_t p, oec_tunedb_t db, const oec_field_desc* in, int n_in,
                            const oec_field_desc* out, int n_out, const int64_t lb[3], const int64_t ub[3],
                            const int64_t halo[3], const double* params, int n_params, int reps, void* cuda_stream,
                            int* from_db) {
  clear_error();
  if (!p || !db || !from_db) return fail(OEC_ERR_INVALID_ARG, "null argument");
  *from_db = 0;
  oec_schedule s{};
  double ms = 0;
  int found = 0;
  int rc = oec_tunedb_find(db, p, in, n_in, out, n_out, lb, ub, &s, &ms, &found);
  if (rc) return rc;
  std::string why;
  if (found && schedule_ok(p->kind, s, why)) {
    p->sched = s;
    *from_db = 1;
    return OEC_OK;
  }
  const int n = oec_program_candidates(p, nullptr, 0);
  if (n <= 0) return n < 0 ? n : fail(OEC_ERR_UNSUPPORTED, "no candidate schedules");
  std::vector<double> times(n);
  int best = -1;
  rc = oec_program_autotune(p, in, n_in, out, n_out, lb, ub, halo, params, n_params, nullptr, 0, reps, cuda_stream,
                            times.data(), &best);
  if (rc) return rc;
  return oec_tunedb_record(db, p, in, n_in, out, n_out, lb, ub, &p->sched, best >= 0 ? times[best] : 0.0);
}
