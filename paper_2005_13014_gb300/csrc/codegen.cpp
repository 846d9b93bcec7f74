// codegen.cpp - generic stencil programs: CUDA C++ generated from the program's
// IR for a schedule, compiled at run time with NVRTC for sm_103a.
//
// Lowering (paper §V-C, §VI): every materialised stage becomes one kernel over
// its inferred range (paper §V-B) writing a temporary in device memory; all
// other stages are inlined into their consumers (paper §V-A): a consumer that
// reads a producer at an offset re-evaluates the producer's body shifted by
// that offset. Within one kernel every (value, offset) pair is evaluated once
// (common subexpression elimination, §V-A). Unrolling by U along k evaluates U
// consecutive levels per thread with one CSE scope, so levels share loads and
// partial results (stencil unrolling, §V-A); a ragged last group of levels is
// shifted down to overlap the previous one (its values are recomputed, and
// rewritten with the same bits), instead of the paper's restriction to
// divisors. Extents, strides and temporary layouts are compile-time constants
// (the paper's size specialisation, §IV), so kernels are specialised per shape.
//
// Fusion modes: OEC_FUSE_INLINE materialises nothing but the outputs;
// OEC_FUSE_NONE materialises every stage (the paper's "original" level);
// OEC_FUSE_PARTIAL materialises stages read at more than two distinct offsets.
#include <cuda_runtime.h>
#include <dlfcn.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <string>
#include <vector>

#include "../../include/oec.h"
#include "api_internal.h"
#include "ir.h"
#include "kernels.h"

namespace oec {
namespace {

// ---- NVRTC, loaded on first use -------------------------------------------
typedef int nvrtcResult_;
typedef struct _nvrtcProgram* nvrtcProgram_;
struct Nvrtc {
  bool ok = false;
  std::string err;
  nvrtcResult_ (*create)(nvrtcProgram_*, const char*, const char*, int, const char* const*, const char* const*);
  nvrtcResult_ (*compile)(nvrtcProgram_, int, const char* const*);
  nvrtcResult_ (*log_size)(nvrtcProgram_, size_t*);
  nvrtcResult_ (*log)(nvrtcProgram_, char*);
  nvrtcResult_ (*cubin_size)(nvrtcProgram_, size_t*);
  nvrtcResult_ (*cubin)(nvrtcProgram_, char*);
  nvrtcResult_ (*destroy)(nvrtcProgram_*);
};

Nvrtc& nvrtc() {
  static Nvrtc n;
  static std::once_flag once;
  std::call_once(once, [] {
    const char* names[] = {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13"};
    void* h = nullptr;
    for (const char* nm : names)
      if ((h = dlopen(nm, RTLD_NOW | RTLD_LOCAL))) break;
    if (!h) {
      n.err = "libnvrtc not found";
      return;
    }
    n.create = (decltype(n.create))dlsym(h, "nvrtcCreateProgram");
    n.compile = (decltype(n.compile))dlsym(h, "nvrtcCompileProgram");
    n.log_size = (decltype(n.log_size))dlsym(h, "nvrtcGetProgramLogSize");
    n.log = (decltype(n.log))dlsym(h, "nvrtcGetProgramLog");
    n.cubin_size = (decltype(n.cubin_size))dlsym(h, "nvrtcGetCUBINSize");
    n.cubin = (decltype(n.cubin))dlsym(h, "nvrtcGetCUBIN");
    n.destroy = (decltype(n.destroy))dlsym(h, "nvrtcDestroyProgram");
    n.ok = n.create && n.compile && n.log_size && n.log && n.cubin_size && n.cubin && n.destroy;
    if (!n.ok) n.err = "libnvrtc lacks a required symbol";
  });
  return n;
}

std::string fmt(const char* f, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, f);
  std::vsnprintf(buf, sizeof buf, f, ap);
  va_end(ap);
  return buf;
}

// ---- plans ----------------------------------------------------------------
struct KernelPlan {
  std::string name;
  Box box;                      // iteration range (logical, relative to lb = 0)
  std::vector<int> stmts;       // statements evaluated and stored by this kernel
  int unroll = 1;
};

struct Layout {
  // temporaries: value id -> (scratch offset, box)
  std::map<int, std::pair<size_t, Box>> tmp;
  size_t bytes = 0;
};

struct Variant {
  int fusion = 0, unroll = 1;
  std::vector<KernelPlan> kernels;
  std::set<int> materialised;   // statement ids
  Layout layout;
  std::vector<cudaKernel_t> fn; // per kernel (after load)
};

struct ShapeKey {
  int64_t ni, nj, nk, sj, sk;
  int arith = 0;   // 1: FP64 programs evaluated in double-float
  int idx64 = 0;   // 1: 64-bit element offsets asked for (OEC_INDEX_64)
  bool operator<(const ShapeKey& o) const {
    return std::tie(ni, nj, nk, sj, sk, arith, idx64) < std::tie(o.ni, o.nj, o.nk, o.sj, o.sk, o.arith, o.idx64);
  }
};

// the double-float arithmetic (csrc/df64.cuh without its includes), for NVRTC
const char* const kDf64Source =
#include "df64_nvrtc.inc"
    ;

struct Module {
  cudaLibrary_t lib = nullptr;
  std::map<std::pair<int, int>, Variant> variants;   // (fusion, unroll)
  int dev = -1;
};

}  // namespace
}  // namespace oec

namespace oec {
std::mutex g_gen_alloc;   // guards creation of a program's generator state
}

struct oec_generic_state {
  std::mutex mu;
  std::map<oec::ShapeKey, std::unique_ptr<oec::Module>> modules;
  ~oec_generic_state() {
    for (auto& m : modules)
      if (m.second->lib) cudaLibraryUnload(m.second->lib);
  }
};

namespace oec {
namespace {

// distinct offsets at which a statement's results are read by its consumers
size_t read_offsets(const Program& p, int stmt) {
  std::set<std::array<int, 3>> offs;
  std::vector<std::pair<int, std::array<int, 3>>> acc;
  for (const Stmt& s : p.stmts) {
    acc.clear();
    if (s.kind == StmtKind::Stage) stmt_accesses(p, s, acc);
    for (auto& a : acc)
      if (p.values[a.first].kind != ValueKind::Input && p.values[a.first].stmt == stmt) offs.insert(a.second);
  }
  return offs.size();
}

bool has_consumer(const Program& p, int value) {
  std::vector<std::pair<int, std::array<int, 3>>> acc;
  for (const Stmt& s : p.stmts) {
    acc.clear();
    if (s.kind == StmtKind::Stage) stmt_accesses(p, s, acc);
    for (auto& a : acc)
      if (a.first == value) return true;
  }
  return false;
}

bool is_output(const Program& p, int value) {
  return std::find(p.outputs.begin(), p.outputs.end(), value) != p.outputs.end();
}

// Code emitter for one kernel: memoised evaluation of (value, offset).
struct Emitter {
  const Program& p;
  const std::vector<Box>& ranges;
  const std::set<int>& mat;          // materialised statement ids (read from temporaries)
  const Layout& lay;
  const ShapeKey& sh;
  const char* T;
  std::string body;
  int next = 0;
  std::map<std::tuple<int, int, int, int>, std::vector<std::string>> stage_memo;   // (stmt, di, dj, dk)
  std::map<std::tuple<int, int, int, int>, std::string> load_memo;               // (value, di, dj, dk)
  int ksize = 0;

  std::string tmpname() { return fmt("t%d", next++); }

  bool df = false;   // compute type is df64 (storage binary64)

  std::string literal(double v) {
    if (df) {
      const float hi = (float)v, lo = (float)(v - (double)hi);
      return fmt("df64{%af, %af}", hi, lo);
    }
    return fmt("((%s)%a)", T, v);
  }

  std::string value(int v, int di, int dj, int dk) {
    const Value& val = p.values[v];
    if (val.kind == ValueKind::Input || mat.count(val.stmt)) {
      auto key = std::make_tuple(v, di, dj, dk);
      auto it = load_memo.find(key);
      if (it != load_memo.end()) return it->second;
      std::string n = tmpname();
      if (val.kind == ValueKind::Input) {
        body += fmt("  const %s %s = cvt_in(__ldg(in%d + (%lldLL)));\n", T, n.c_str(), val.index,
                    (long long)di + (long long)dj * sh.sj + (long long)dk * sh.sk);
      } else {
        const Box& b = lay.tmp.at(v).second;
        const long long tj = b.hi[0] - b.lo[0], tk = tj * (b.hi[1] - b.lo[1]);
        body += fmt("  const %s %s = tp%d[%lldLL];\n", T, n.c_str(), v, (long long)di + dj * tj + dk * tk);
      }
      load_memo[key] = n;
      return n;
    }
    return stage(val.stmt, di, dj, dk)[val.index];
  }

  const std::vector<std::string>& stage(int si, int di, int dj, int dk) {
    auto key = std::make_tuple(si, di, dj, dk);
    auto it = stage_memo.find(key);
    if (it != stage_memo.end()) return it->second;
    const Stmt& st = p.stmts[si];
    std::map<int, std::string> lets;
    for (auto& l : st.lets) lets[l.first] = expr(l.second, di, dj, dk, lets);
    std::vector<std::string> res;
    for (int r : st.rets) res.push_back(expr(r, di, dj, dk, lets));
    return stage_memo[key] = res;
  }

  std::string expr(int id, int di, int dj, int dk, const std::map<int, std::string>& lets) {
    const Expr& e = p.pool[id];
    auto sub = [&](int c) { return expr(c, di, dj, dk, lets); };
    std::string n;
    switch (e.op) {
      case Op::Num: return literal(e.num);
      case Op::Acc: return value(e.ref, di + e.off[0], dj + e.off[1], dk + e.off[2]);
      case Op::Let: return lets.at(e.ref);
      case Op::Param: return fmt("P%d", e.ref);
      case Op::KPos: return df ? fmt("df64{(float)(k + %d), 0.0f}", dk) : fmt("((%s)(k + %d))", T, dk);
      case Op::KSize: return literal((double)sh.nk);
      default: break;
    }
    n = tmpname();
    switch (e.op) {
      case Op::Neg: body += fmt("  const %s %s = -%s;\n", T, n.c_str(), sub(e.a).c_str()); break;
      case Op::Abs: body += fmt("  const %s %s = cabs_(%s);\n", T, n.c_str(), sub(e.a).c_str()); break;
      case Op::Add:
      case Op::Sub:
      case Op::Mul:
      case Op::Div: {
        const char* op = e.op == Op::Add ? "+" : e.op == Op::Sub ? "-" : e.op == Op::Mul ? "*" : "/";
        std::string a = sub(e.a), b = sub(e.b);
        body += fmt("  const %s %s = %s %s %s;\n", T, n.c_str(), a.c_str(), op, b.c_str());
        break;
      }
      case Op::Min:
      case Op::Max: {
        std::string a = sub(e.a), b = sub(e.b);
        body += fmt("  const %s %s = %s(%s, %s);\n", T, n.c_str(), e.op == Op::Min ? "cmin_" : "cmax_", a.c_str(), b.c_str());
        break;
      }
      case Op::Sel: {
        static const char* rel[] = {">", "<", ">=", "<="};
        std::string x = sub(e.a), y = sub(e.b), a = sub(e.c), b = sub(e.d);
        body += fmt("  const %s %s = (%s %s %s) ? %s : %s;\n", T, n.c_str(), x.c_str(), rel[int(e.rel)], y.c_str(),
                    a.c_str(), b.c_str());
        break;
      }
      default: break;
    }
    return n;
  }
};

Variant plan_variant(const Program& p, const std::vector<Box>& ranges, const ShapeKey& sh, int fusion, int unroll,
                     size_t es) {
  Variant v;
  v.fusion = fusion;
  v.unroll = unroll;
  for (int si = 0; si < (int)p.stmts.size(); ++si) {
    const Stmt& st = p.stmts[si];
    if (!ranges[st.results[0]].valid) continue;       // dead
    bool feeds = false;
    for (int r : st.results) feeds |= has_consumer(p, r);
    if (!feeds) continue;                            // output-only: evaluated by the output kernel
    if (fusion == OEC_FUSE_NONE || (fusion == OEC_FUSE_PARTIAL && read_offsets(p, si) > 2)) v.materialised.insert(si);
  }
  // temporaries of materialised results that other stages read
  size_t off = 0;
  for (int si : v.materialised)
    for (int r : p.stmts[si].results) {
      if (!has_consumer(p, r)) continue;
      const Box& b = ranges[r];
      v.layout.tmp[r] = {off, b};
      off = align_up(off + es * (size_t)b.volume(), 256);
    }
  v.layout.bytes = off;
  auto clamp_unroll = [&](const Box& b) { return (int)std::max<int64_t>(1, std::min<int64_t>(unroll, b.hi[2] - b.lo[2])); };
  for (int si : v.materialised) {
    KernelPlan kp;
    kp.name = fmt("k_f%d_u%d_s%d", fusion, unroll, si);
    kp.box = ranges[p.stmts[si].results[0]];
    kp.stmts = {si};
    kp.unroll = clamp_unroll(kp.box);
    v.kernels.push_back(kp);
  }
  // outputs not already written by a materialised kernel
  KernelPlan out;
  out.name = fmt("k_f%d_u%d_out", fusion, unroll);
  for (int d = 0; d < 3; ++d) { out.box.lo[d] = 0; out.box.hi[d] = d == 0 ? sh.ni : d == 1 ? sh.nj : sh.nk; }
  out.box.valid = true;
  for (int o : p.outputs) {
    const int si = p.values[o].stmt;
    if (!v.materialised.count(si) && std::find(out.stmts.begin(), out.stmts.end(), si) == out.stmts.end())
      out.stmts.push_back(si);
  }
  out.unroll = clamp_unroll(out.box);
  if (!out.stmts.empty()) v.kernels.push_back(out);
  return v;
}

// true when every element offset the generated kernels form from a field's
// domain corner (points of the inferred ranges) fits in an int32
bool field_offsets_fit_int32(const std::vector<Box>& ranges, const ShapeKey& sh) {
  if (sh.sj >= INT32_MAX || sh.sk >= INT32_MAX) return false;
  const int64_t s[3] = {1, sh.sj, sh.sk};
  int64_t lo[3] = {0, 0, 0}, hi[3] = {sh.ni, sh.nj, sh.nk};
  for (const Box& b : ranges)
    if (b.valid)
      for (int d = 0; d < 3; ++d) { lo[d] = std::min(lo[d], b.lo[d]); hi[d] = std::max(hi[d], b.hi[d]); }
  int64_t m = 0;
  for (int d = 0; d < 3; ++d) m += std::max(std::abs(lo[d]), std::abs(hi[d])) * s[d];
  return m < INT32_MAX;
}

// o32: the element offsets (the thread's point in the fields and in the
// temporaries) are computed in 32-bit ints, else in 64-bit
std::string kernel_source(const Program& p, const std::vector<Box>& ranges, const Variant& v, const KernelPlan& kp,
                          const ShapeKey& sh, const char* T, bool o32) {
  std::set<int> mat_except_self = v.materialised;
  for (int si : kp.stmts) mat_except_self.erase(si);
  Emitter e{p, ranges, mat_except_self, v.layout, sh, T};
  e.df = sh.arith == 1;
  const Box& b = kp.box;
  const int64_t bni = b.hi[0] - b.lo[0], bnj = b.hi[1] - b.lo[1], bnk = b.hi[2] - b.lo[2];
  std::string src;
  src += fmt("extern \"C\" __global__ void %s(Args a) {\n", kp.name.c_str());
  src += "  const int ii = blockIdx.x * blockDim.x + threadIdx.x, jj = blockIdx.y * blockDim.y + threadIdx.y;\n";
  src += fmt("  int kk = blockIdx.z * %d;\n", kp.unroll);
  src += fmt("  if (ii >= %lld || jj >= %lld) return;\n", (long long)bni, (long long)bnj);
  src += fmt("  if (kk > %lld) kk = %lld;\n", (long long)(bnk - kp.unroll), (long long)(bnk - kp.unroll));
  src += fmt("  const int i = ii + (%lld), j = jj + (%lld), k = kk + (%lld);\n", (long long)b.lo[0], (long long)b.lo[1],
             (long long)b.lo[2]);
  if (o32)
    src += fmt("  const int fo = k * %lld + j * %lld + i;\n", (long long)sh.sk, (long long)sh.sj);
  else
    src += "  const long long fo = (long long)k * " + fmt("%lldLL", (long long)sh.sk) + " + (long long)j * " +
           fmt("%lldLL", (long long)sh.sj) + " + i;\n";
  for (size_t x = 0; x < p.inputs.size(); ++x)
    src += fmt("  const S_* __restrict__ in%zu = a.in[%zu] + fo;\n", x, x);
  for (size_t x = 0; x < p.params.size(); ++x) src += fmt("  const %s P%zu = cvt_in(a.prm[%zu]);\n", T, x, x);
  for (auto& t : v.layout.tmp) {
    const Box& tb = t.second.second;
    const long long tj = tb.hi[0] - tb.lo[0], tk = tj * (tb.hi[1] - tb.lo[1]);
    if (o32)
      src += fmt("  %s* __restrict__ tp%d = (%s*)(a.scratch + %zuULL) + ((k - (%lld)) * %lld + (j - (%lld)) * %lld + "
                 "(i - (%lld)));\n",
                 T, t.first, T, t.second.first, (long long)tb.lo[2], tk, (long long)tb.lo[1], tj, (long long)tb.lo[0]);
    else
      src += fmt("  %s* __restrict__ tp%d = (%s*)(a.scratch + %zuULL) + ((long long)(k - (%lld)) * %lldLL + "
                 "(long long)(j - (%lld)) * %lldLL + (i - (%lld)));\n",
                 T, t.first, T, t.second.first, (long long)tb.lo[2], tk, (long long)tb.lo[1], tj, (long long)tb.lo[0]);
  }
  for (int u = 0; u < kp.unroll; ++u) {
    for (int si : kp.stmts) {
      const std::vector<std::string> res = e.stage(si, 0, 0, u);
      const Stmt& st = p.stmts[si];
      for (size_t r = 0; r < st.results.size(); ++r) {
        const int val = st.results[r];
        if (v.layout.tmp.count(val)) {
          const Box& tb = v.layout.tmp.at(val).second;
          const long long tj = tb.hi[0] - tb.lo[0], tk = tj * (tb.hi[1] - tb.lo[1]);
          e.body += fmt("  tp%d[%lldLL] = %s;\n", val, (long long)u * tk, res[r].c_str());
        }
        for (size_t o = 0; o < p.outputs.size(); ++o)
          if (p.outputs[o] == val) {
            e.body += fmt("  if (i >= 0 && i < %lld && j >= 0 && j < %lld && k + %d >= 0 && k + %d < %lld)\n",
                          (long long)sh.ni, (long long)sh.nj, u, u, (long long)sh.nk);
            e.body += fmt("    a.out[%zu][fo + %lldLL] = cvt_out(%s);\n", o, (long long)u * sh.sk, res[r].c_str());
          }
      }
    }
  }
  src += e.body;
  src += "}\n";
  return src;
}

std::string module_source(oec_program* prog, const ShapeKey& sh, const std::vector<Box>& ranges, Module& m) {
  const Program& p = prog->ir;
  const char* S = prog->dtype == OEC_F64 ? "double" : "float";
  const bool df = sh.arith == 1;
  const char* T = df ? "df64" : S;   // compute type
  const size_t es = elem_size(prog->dtype);   // df64 pairs are 8 bytes, as binary64
  std::string src;
  if (df) {
    src += kDf64Source;
    src += "using namespace oec;\n"
           "__device__ __forceinline__ df64 cvt_in(double x) { return df_from_double(x); }\n"
           "__device__ __forceinline__ double cvt_out(df64 x) { return df_to_double(x); }\n"
           "__device__ __forceinline__ bool operator<(df64 a, df64 b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }\n"
           "__device__ __forceinline__ bool operator>(df64 a, df64 b) { return b < a; }\n"
           "__device__ __forceinline__ bool operator<=(df64 a, df64 b) { return !(b < a); }\n"
           "__device__ __forceinline__ bool operator>=(df64 a, df64 b) { return !(a < b); }\n"
           "__device__ __forceinline__ df64 cabs_(df64 a) { return df_abs(a); }\n"
           "__device__ __forceinline__ df64 cmin_(df64 a, df64 b) { return b < a ? b : a; }\n"
           "__device__ __forceinline__ df64 cmax_(df64 a, df64 b) { return a < b ? b : a; }\n";
  } else {
    src += fmt("__device__ __forceinline__ %s cvt_in(%s x) { return x; }\n", S, S);
    src += fmt("__device__ __forceinline__ %s cvt_out(%s x) { return x; }\n", S, S);
    src += fmt("__device__ __forceinline__ %s cabs_(%s a) { return fabs(a); }\n", S, S);
    src += fmt("__device__ __forceinline__ %s cmin_(%s a, %s b) { return fmin(a, b); }\n", S, S, S);
    src += fmt("__device__ __forceinline__ %s cmax_(%s a, %s b) { return fmax(a, b); }\n", S, S, S);
  }
  src += fmt("typedef %s S_;\n", S);
  // layout shared with the host; the scalar parameters travel by value with
  // every launch (a launch captured into a CUDA graph keeps its own values)
  src += "struct Args { const S_* in[16]; S_* out[8]; char* scratch; double prm[16]; };\n";
  const bool f32 = !sh.idx64 && field_offsets_fit_int32(ranges, sh);
  for (int fusion : {OEC_FUSE_INLINE, OEC_FUSE_NONE, OEC_FUSE_PARTIAL})
    for (int unroll : {1, 2, 4}) {
      Variant v = plan_variant(p, ranges, sh, fusion, unroll, es);
      const bool o32 = f32 && v.layout.bytes / es < (size_t)INT32_MAX;
      for (const KernelPlan& kp : v.kernels) src += kernel_source(p, ranges, v, kp, sh, T, o32);
      m.variants[{fusion, unroll}] = std::move(v);
    }
  return src;
}

int nvrtc_compile(const std::string& src, std::vector<char>& cubin) {
  if (fault_injected("compile")) return fail(OEC_ERR_COMPILE, "compile failure injected by OEC_FAULT=compile");
  Nvrtc& nv = nvrtc();
  if (!nv.ok) return fail(OEC_ERR_COMPILE, "%s", nv.err.c_str());
  nvrtcProgram_ np = nullptr;
  if (nv.create(&np, src.c_str(), "oec_generated.cu", 0, nullptr, nullptr) != 0)
    return fail(OEC_ERR_COMPILE, "nvrtcCreateProgram failed");
  const char* opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "--fmad=true", "-default-device"};
  const int rc = nv.compile(np, 4, opts);
  if (rc != 0) {
    size_t ls = 0;
    nv.log_size(np, &ls);
    std::string log(ls, '\0');
    nv.log(np, &log[0]);
    nv.destroy(&np);
    return fail(OEC_ERR_COMPILE, "NVRTC: %.400s", log.c_str());
  }
  size_t cs = 0;
  nv.cubin_size(np, &cs);
  cubin.resize(cs);
  nv.cubin(np, cubin.data());
  nv.destroy(&np);
  return OEC_OK;
}

int compile_module(oec_program* prog, const ShapeKey& sh, const std::vector<Box>& ranges, Module& m) {
  const std::string src = module_source(prog, sh, ranges, m);
  std::vector<char> cubin;
  int rc = nvrtc_compile(src, cubin);
  if (rc) return rc;
  cudaError_t e = cudaLibraryLoadData(&m.lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
  if (e != cudaSuccess) return cuda_fail(e, "cudaLibraryLoadData");
  for (auto& kv : m.variants)
    for (const KernelPlan& kp : kv.second.kernels) {
      cudaKernel_t k = nullptr;
      e = cudaLibraryGetKernel(&k, m.lib, kp.name.c_str());
      if (e != cudaSuccess) return cuda_fail(e, "cudaLibraryGetKernel");
      kv.second.fn.push_back(k);
    }
  cudaGetDevice(&m.dev);
  return OEC_OK;
}

// Per-point counts of one schedule variant, from a dry run of the emitter:
// loads, arithmetic temporaries and stores of every kernel, weighted by the
// kernel's iteration volume over the domain volume and divided by the unroll.
struct VariantStats {
  double loads = 0, ops = 0, stores = 0, temp_bytes = 0, kernels = 0, materialised = 0, max_blocks = 0;
};

VariantStats variant_stats(const Program& p, const std::vector<Box>& ranges, const ShapeKey& sh, int fusion, int unroll,
                           size_t es, int ti, int tj) {
  VariantStats st;
  Variant v = plan_variant(p, ranges, sh, fusion, unroll, es);
  const double dom = double(sh.ni) * sh.nj * sh.nk;
  for (const KernelPlan& kp : v.kernels) {
    std::set<int> mat = v.materialised;
    for (int si : kp.stmts) mat.erase(si);
    Emitter e{p, ranges, mat, v.layout, sh, "float"};
    int stores = 0;
    for (int u = 0; u < kp.unroll; ++u)
      for (int si : kp.stmts) {
        e.stage(si, 0, 0, u);
        for (int r : p.stmts[si].results) stores += (v.layout.tmp.count(r) ? 1 : 0) + (is_output(p, r) ? 1 : 0);
      }
    const double w = double(kp.box.volume()) / dom / kp.unroll;
    st.loads += w * e.load_memo.size();
    st.ops += w * (e.next - (int)e.load_memo.size());
    st.stores += w * stores;
    const double blocks = std::ceil(double(kp.box.hi[0] - kp.box.lo[0]) / ti) *
                          std::ceil(double(kp.box.hi[1] - kp.box.lo[1]) / tj) *
                          std::ceil(double(kp.box.hi[2] - kp.box.lo[2]) / kp.unroll);
    st.max_blocks = std::max(st.max_blocks, blocks);
  }
  st.kernels = (double)v.kernels.size();
  st.temp_bytes = double(v.layout.bytes) / dom;
  st.materialised = (double)v.materialised.size();
  return st;
}

int depth_of(const Program& p) {
  std::vector<int> d(p.stmts.size(), 1);
  std::vector<std::pair<int, std::array<int, 3>>> acc;
  int best = 0;
  for (size_t si = 0; si < p.stmts.size(); ++si) {
    acc.clear();
    if (p.stmts[si].kind == StmtKind::Stage) stmt_accesses(p, p.stmts[si], acc);
    for (auto& a : acc)
      if (p.values[a.first].kind != ValueKind::Input) d[si] = std::max(d[si], d[p.values[a.first].stmt] + 1);
    best = std::max(best, d[si]);
  }
  return best;
}

}  // namespace

constexpr int kNumFeatures = 42;

int program_features(oec_program* prog, const int64_t ext[3], int64_t sj, int64_t sk, const oec_schedule& s,
                     float* out) {
  const Program& p = prog->ir;
  const ShapeKey sh{ext[0], ext[1], ext[2], sj, sk};
  const int64_t zlb[3] = {0, 0, 0}, zub[3] = {ext[0], ext[1], ext[2]};
  std::vector<Box> ranges;
  std::string err;
  if (!infer_ranges(p, zlb, zub, ranges, err)) return fail(OEC_ERR_SHAPE, "%s", err.c_str());
  const size_t es = elem_size(prog->dtype);
  int n_access = 0, n_arith = 0, n_sel = 0, n_mm = 0, n_div = 0, md[3] = {0, 0, 0};
  for (const Expr& e : p.pool) {
    switch (e.op) {
      case Op::Acc:
        ++n_access;
        for (int d = 0; d < 3; ++d) md[d] = std::max(md[d], std::abs(e.off[d]));
        break;
      case Op::Sel: ++n_sel; ++n_arith; break;
      case Op::Min: case Op::Max: ++n_mm; ++n_arith; break;
      case Op::Div: ++n_div; ++n_arith; break;
      case Op::Neg: case Op::Abs: case Op::Add: case Op::Sub: case Op::Mul: ++n_arith; break;
      default: break;
    }
  }
  double halo[3] = {0, 0, 0}, amp = 0;
  const double dom = double(ext[0]) * ext[1] * ext[2];
  for (int v : p.inputs) {
    const Box& b = ranges[v];
    if (!b.valid) continue;
    for (int d = 0; d < 3; ++d) halo[d] = std::max(halo[d], 0.5 * double((zlb[d] - b.lo[d]) + (b.hi[d] - zub[d])));
    amp += double(b.volume()) / dom;
  }
  amp /= std::max<size_t>(1, p.inputs.size());
  const VariantStats vs = variant_stats(p, ranges, sh, s.fusion, s.unroll, es, s.tile_i, s.tile_j);
  const VariantStats v0 = variant_stats(p, ranges, sh, OEC_FUSE_INLINE, 1, es, s.tile_i, s.tile_j);
  const VariantStats vn = variant_stats(p, ranges, sh, OEC_FUSE_NONE, 1, es, s.tile_i, s.tile_j);
  auto l2 = [](double x) { return (float)std::log2(std::max(1.0, x)); };
  const double eff_i = double(ext[0]) / (std::ceil(double(ext[0]) / s.tile_i) * s.tile_i);
  const double eff_j = double(ext[1]) / (std::ceil(double(ext[1]) / s.tile_j) * s.tile_j);
  const double bytes_pp = es * (amp * p.inputs.size() + p.outputs.size() + 2.0 * vs.temp_bytes / es);
  float f[kNumFeatures] = {
      (float)p.stmts.size(), (float)p.inputs.size(), (float)p.outputs.size(), (float)n_access, (float)n_arith,
      (float)n_sel, (float)n_mm, (float)n_div, (float)md[0], (float)md[1], (float)md[2], (float)depth_of(p),
      (float)halo[0], (float)halo[1], (float)halo[2], (float)amp, l2(ext[0]), l2(ext[1]), l2(ext[2]), l2(dom),
      (float)es, s.fusion == OEC_FUSE_INLINE ? 1.f : 0.f, s.fusion == OEC_FUSE_NONE ? 1.f : 0.f,
      s.fusion == OEC_FUSE_PARTIAL ? 1.f : 0.f, l2(s.unroll), l2(s.tile_i), l2(s.tile_j), l2(s.tile_i * s.tile_j),
      (float)vs.kernels, (float)vs.loads, (float)vs.ops, (float)vs.stores, (float)vs.temp_bytes, l2(vs.max_blocks),
      (float)eff_i, (float)eff_j, (float)bytes_pp, (float)v0.ops, (float)(vs.ops / std::max(1.0, vn.ops)),
      (float)vs.materialised, (float)(vs.max_blocks / 152.0), l2(vs.ops * dom)};
  for (int x = 0; x < kNumFeatures; ++x) out[x] = f[x];
  return OEC_OK;
}

// the compiled module of a program for one shape (compiled on first use)
int get_module(oec_program* p, const ShapeKey& key, Module** out) {
  {
    std::lock_guard<std::mutex> lock(g_gen_alloc);
    if (!p->gen) p->gen = new (std::nothrow) oec_generic_state();
  }
  if (!p->gen) return fail(OEC_ERR_INVALID_ARG, "out of host memory");
  std::lock_guard<std::mutex> lock(p->gen->mu);
  auto it = p->gen->modules.find(key);
  if (it == p->gen->modules.end()) {
    const int64_t zlb[3] = {0, 0, 0}, zub[3] = {key.ni, key.nj, key.nk};
    std::vector<Box> ranges;
    std::string err;
    if (!infer_ranges(p->ir, zlb, zub, ranges, err)) return fail(OEC_ERR_SHAPE, "%s", err.c_str());
    std::unique_ptr<Module> nm(new Module());
    int rc = compile_module(p, key, ranges, *nm);
    if (rc) return rc;
    it = p->gen->modules.emplace(key, std::move(nm)).first;
  }
  *out = it->second.get();
  return OEC_OK;
}

bool generic_schedule_ok(const oec_schedule& s, std::string& why) {
  if (s.fusion != OEC_FUSE_INLINE && s.fusion != OEC_FUSE_NONE && s.fusion != OEC_FUSE_PARTIAL) {
    why = "fusion must be OEC_FUSE_INLINE, OEC_FUSE_NONE or OEC_FUSE_PARTIAL";
    return false;
  }
  if (s.unroll != 1 && s.unroll != 2 && s.unroll != 4) { why = "unroll (along k) must be 1, 2 or 4"; return false; }
  if (s.tile_i < 1 || s.tile_j < 1 || s.tile_i * s.tile_j > 1024 || s.tile_i > 1024) {
    why = "tile_i * tile_j must be in [1, 1024]";
    return false;
  }
  if (s.arith != 0 && s.arith != 1) {
    why = "generated kernels: arith 0 (the dtype's own) or 1 (double-float, FP64 programs)";
    return false;
  }
  return true;
}

void generic_release(oec_program* p) {
  delete p->gen;
  p->gen = nullptr;
}

int generic_apply(oec_program* p, const oec_field_desc* in, const oec_field_desc* out, const int64_t lb[3],
                  const int64_t ub[3], const double* params, cudaStream_t st) {
  const Program& ir = p->ir;
  for (const Stmt& s : ir.stmts)
    if (s.kind == StmtKind::Column) return fail(OEC_ERR_UNSUPPORTED, "generated kernels do not solve columns");
  const size_t es = elem_size(p->dtype);
  const int n_in = (int)ir.inputs.size(), n_out = (int)ir.outputs.size();
  const int64_t sj = out[0].stride[1], sk = out[0].stride[2];
  for (int x = 0; x < n_in + n_out; ++x) {
    const oec_field_desc& f = x < n_in ? in[x] : out[x - n_in];
    if (f.ndim != 3 || f.stride[1] != sj || f.stride[2] != sk)
      return fail(OEC_ERR_UNSUPPORTED, "generated kernels need 3-D fields with equal j/k strides (field %d differs)", x);
  }
  if (n_in > 16 || n_out > 8) return fail(OEC_ERR_UNSUPPORTED, "at most 16 inputs and 8 outputs");
  if (p->sched.arith == 1 && p->dtype != OEC_F64)
    return fail(OEC_ERR_UNSUPPORTED, "double-float generated kernels are for FP64 programs");
  const ShapeKey key{ub[0] - lb[0], ub[1] - lb[1], ub[2] - lb[2], sj, sk, p->sched.arith,
                     p->sched.index_bits == OEC_INDEX_64 ? 1 : 0};
  Module* m = nullptr;
  int rc = get_module(p, key, &m);
  if (rc) return rc;
  const Variant& v = m->variants.at({p->sched.fusion, p->sched.unroll});
  rc = ensure_scratch(p, v.layout.bytes);
  if (rc) return rc;
  if (ir.params.size() > 16) return fail(OEC_ERR_UNSUPPORTED, "at most 16 scalar parameters");
  struct Args {   // the generated kernels' argument, passed by value
    const void* in[16];
    void* out[8];
    char* scratch;
    double prm[16];
  } args{};
  for (size_t x = 0; x < ir.params.size(); ++x) args.prm[x] = params[x];
  auto base_at = [&](const oec_field_desc& f) {
    int64_t off = 0;
    for (int d = 0; d < 3; ++d) off += (f.origin[d] + lb[d]) * f.stride[d];
    return (char*)f.data + off * (int64_t)es;
  };
  for (int x = 0; x < n_in; ++x) args.in[x] = base_at(in[x]);
  for (int x = 0; x < n_out; ++x) args.out[x] = base_at(out[x]);
  args.scratch = (char*)p->scratch;
  void* kargs[] = {&args};
  for (size_t x = 0; x < v.kernels.size(); ++x) {
    const KernelPlan& kp = v.kernels[x];
    const Box& b = kp.box;
    const int64_t bni = b.hi[0] - b.lo[0], bnj = b.hi[1] - b.lo[1], bnk = b.hi[2] - b.lo[2];
    dim3 blk(std::min<int>(p->sched.tile_i, 1024), p->sched.tile_j);
    dim3 grd((unsigned)((bni + blk.x - 1) / blk.x), (unsigned)((bnj + blk.y - 1) / blk.y),
             (unsigned)((bnk + kp.unroll - 1) / kp.unroll));
    cudaError_t e = cudaLaunchKernel((const void*)v.fn[x], grd, blk, kargs, 0, st);
    if (e != cudaSuccess) return cuda_fail(e, "generated kernel launch");
    launched(st);
  }
  return OEC_OK;
}

}  // namespace oec

using namespace oec;

extern "C" int oec_program_features(oec_program_t p, const int64_t extent[3], int64_t sj, int64_t sk,
                                    const oec_schedule* s, float* out, int cap) {
  clear_error();
  if (!p || !extent || !s) return fail(OEC_ERR_INVALID_ARG, "null argument");
  if (!out) return kNumFeatures;
  if (cap < kNumFeatures) return fail(OEC_ERR_INVALID_ARG, "need room for %d features", kNumFeatures);
  for (const Stmt& st : p->ir.stmts)
    if (st.kind == StmtKind::Column) return fail(OEC_ERR_UNSUPPORTED, "features describe generated programs");
  if (extent[0] < 1 || extent[1] < 1 || extent[2] < 1 || sj < extent[0] || sk < sj)
    return fail(OEC_ERR_INVALID_ARG, "bad extent or strides");
  std::string why;
  if (!generic_schedule_ok(*s, why)) return fail(OEC_ERR_UNSUPPORTED, "schedule: %s", why.c_str());
  int rc = program_features(p, extent, sj, sk, *s, out);
  return rc ? rc : kNumFeatures;
}

extern "C" int oec_program_prepare(oec_program_t p, const int64_t extent[3], int64_t sj, int64_t sk) {
  clear_error();
  if (!p || !extent) return fail(OEC_ERR_INVALID_ARG, "null argument");
  if (p->kind != OEC_KIND_GENERIC) return OEC_OK;   // hand-written kernels need no preparation
  for (const Stmt& s : p->ir.stmts)
    if (s.kind == StmtKind::Column) return fail(OEC_ERR_UNSUPPORTED, "generated kernels do not solve columns");
  if (extent[0] < 1 || extent[1] < 1 || extent[2] < 1 || sj < extent[0] || sk < sj)
    return fail(OEC_ERR_INVALID_ARG, "bad extent or strides");
  Module* m = nullptr;
  const int arith = p->dtype == OEC_F64 && p->sched.arith == 1 ? 1 : 0;
  return get_module(p, ShapeKey{extent[0], extent[1], extent[2], sj, sk, arith, p->sched.index_bits == OEC_INDEX_64 ? 1 : 0},
                    &m);
}

extern "C" int oec_program_codegen(oec_program_t p, const int64_t extent[3], int64_t sj, int64_t sk, int compile,
                                   char* buf, int64_t cap, int64_t* len) {
  clear_error();
  if (!p || !extent) return fail(OEC_ERR_INVALID_ARG, "null argument");
  for (const Stmt& s : p->ir.stmts)
    if (s.kind == StmtKind::Column) return fail(OEC_ERR_UNSUPPORTED, "generated kernels do not solve columns");
  if (extent[0] < 1 || extent[1] < 1 || extent[2] < 1 || sj < extent[0] || sk < sj)
    return fail(OEC_ERR_INVALID_ARG, "bad extent or strides");
  const ShapeKey key{extent[0], extent[1], extent[2], sj, sk, p->dtype == OEC_F64 && p->sched.arith == 1 ? 1 : 0,
                     p->sched.index_bits == OEC_INDEX_64 ? 1 : 0};
  const int64_t zlb[3] = {0, 0, 0}, zub[3] = {extent[0], extent[1], extent[2]};
  std::vector<Box> ranges;
  std::string err;
  if (!infer_ranges(p->ir, zlb, zub, ranges, err)) return fail(OEC_ERR_SHAPE, "%s", err.c_str());
  Module m;
  const std::string src = module_source(p, key, ranges, m);
  if (len) *len = (int64_t)src.size();
  if (buf && cap > 0) {
    const size_t n = std::min<size_t>(src.size(), (size_t)cap - 1);
    std::memcpy(buf, src.data(), n);
    buf[n] = 0;
  }
  if (compile) {
    std::vector<char> cubin;
    return nvrtc_compile(src, cubin);
  }
  return OEC_OK;
}
