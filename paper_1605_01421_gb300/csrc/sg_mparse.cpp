// sg_mparse.cpp -- models from transition strings (Sec. 3.5, the model
// parser): "LHS -> propensity -> RHS" is turned into a column of the
// state-change matrix S, a row of the dependency graph G and CUDA code for the
// propensity; the code is compiled at run time with NVRTC for sm_103a
// together with the engine's day and event kernels (the generated
// ModelTraits<SG_GENERIC>), the GPU counterpart of compiling the generated C
// code and loading it.
//
// Grammar.  LHS and RHS are "@" (the empty set) or compartment names joined
// by "+", a name optionally preceded by "k*" (k individuals).  A propensity
// is an expression over compartment names (the node's counts as double),
// global-data names, decimal numbers, + - * /, unary minus and plus, and
// parentheses; * and / bind tighter than + and -, operators group left to
// right.  Every operation is one IEEE double operation in that grouping (the
// kernels are compiled without contraction).  Numbers become the nearest
// double (strtod) and are emitted as exact hexadecimal literals.
#include <cuda_runtime.h>
#include <dlfcn.h>
#include <nvrtc.h>

#include <cctype>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "sg_mparse.h"

namespace sg {
namespace {

struct Node {
  enum Kind { NUM, COMP, GD, NEG, BIN } kind;
  double num = 0.0;
  int index = 0;
  char op = 0;
  std::unique_ptr<Node> a, b;
};

struct Lexer {
  const char *s;
  size_t i = 0;
  explicit Lexer(const char *text) : s(text) {}
  void skip() {
    while (s[i] && std::isspace((unsigned char)s[i])) ++i;
  }
  bool at_end() {
    skip();
    return s[i] == 0;
  }
  char peek() {
    skip();
    return s[i];
  }
};

bool name_start(char c) { return std::isalpha((unsigned char)c) || c == '_' || c == '.'; }
bool name_char(char c) { return std::isalnum((unsigned char)c) || c == '_' || c == '.'; }

class Parser {
 public:
  Parser(const char *text, const std::vector<std::string> &comps,
         const std::vector<std::string> &gnames)
      : lx_(text), comps_(comps), gnames_(gnames) {}

  std::unique_ptr<Node> parse(std::string &err) {
    std::unique_ptr<Node> e = sum();
    if (e && !lx_.at_end()) fail(std::string("unexpected '") + lx_.peek() + "'");
    if (!err_.empty()) {
      err = err_;
      return nullptr;
    }
    return e;
  }

 private:
  Lexer lx_;
  const std::vector<std::string> &comps_, &gnames_;
  std::string err_;

  void fail(const std::string &m) {
    if (err_.empty()) err_ = m;
  }

  std::unique_ptr<Node> bin(char op, std::unique_ptr<Node> a, std::unique_ptr<Node> b) {
    auto n = std::make_unique<Node>();
    n->kind = Node::BIN;
    n->op = op;
    n->a = std::move(a);
    n->b = std::move(b);
    return n;
  }

  std::unique_ptr<Node> sum() {
    std::unique_ptr<Node> e = product();
    while (err_.empty() && (lx_.peek() == '+' || lx_.peek() == '-')) {
      const char op = lx_.s[lx_.i++];
      e = bin(op, std::move(e), product());
    }
    return e;
  }

  std::unique_ptr<Node> product() {
    std::unique_ptr<Node> e = unary();
    while (err_.empty() && (lx_.peek() == '*' || lx_.peek() == '/')) {
      const char op = lx_.s[lx_.i++];
      e = bin(op, std::move(e), unary());
    }
    return e;
  }

  std::unique_ptr<Node> unary() {
    const char c = lx_.peek();
    if (c == '-') {
      ++lx_.i;
      auto n = std::make_unique<Node>();
      n->kind = Node::NEG;
      n->a = unary();
      return n;
    }
    if (c == '+') {
      ++lx_.i;
      return unary();
    }
    return primary();
  }

  std::unique_ptr<Node> primary() {
    const char c = lx_.peek();
    auto n = std::make_unique<Node>();
    if (std::isdigit((unsigned char)c) || (c == '.' && std::isdigit((unsigned char)lx_.s[lx_.i + 1]))) {
      // decimal number: digits [. digits] [e [+-] digits]
      size_t j = lx_.i;
      while (std::isdigit((unsigned char)lx_.s[j])) ++j;
      if (lx_.s[j] == '.') {
        ++j;
        while (std::isdigit((unsigned char)lx_.s[j])) ++j;
      }
      if (lx_.s[j] == 'e' || lx_.s[j] == 'E') {
        size_t k = j + 1;
        if (lx_.s[k] == '+' || lx_.s[k] == '-') ++k;
        if (std::isdigit((unsigned char)lx_.s[k])) {
          while (std::isdigit((unsigned char)lx_.s[k])) ++k;
          j = k;
        }
      }
      const std::string text(lx_.s + lx_.i, j - lx_.i);
      lx_.i = j;
      n->kind = Node::NUM;
      n->num = std::strtod(text.c_str(), nullptr);
      return n;
    }
    if (name_start(c)) {
      size_t j = lx_.i;
      while (name_char(lx_.s[j])) ++j;
      const std::string name(lx_.s + lx_.i, j - lx_.i);
      lx_.i = j;
      for (size_t p = 0; p < comps_.size(); ++p)
        if (comps_[p] == name) {
          n->kind = Node::COMP;
          n->index = (int)p;
          return n;
        }
      for (size_t q = 0; q < gnames_.size(); ++q)
        if (gnames_[q] == name) {
          n->kind = Node::GD;
          n->index = (int)q;
          return n;
        }
      fail("unknown name '" + name + "'");
      return nullptr;
    }
    if (c == '(') {
      ++lx_.i;
      std::unique_ptr<Node> e = sum();
      if (lx_.peek() != ')') {
        fail("missing ')'");
        return nullptr;
      }
      ++lx_.i;
      return e;
    }
    fail(c ? std::string("unexpected '") + c + "'" : std::string("unexpected end"));
    return nullptr;
  }
};

void reads(const Node *n, std::vector<char> &acc) {
  if (!n) return;
  if (n->kind == Node::COMP) acc[n->index] = 1;
  reads(n->a.get(), acc);
  reads(n->b.get(), acc);
}

std::string code(const Node *n) {
  char buf[64];
  switch (n->kind) {
    case Node::NUM:
      std::snprintf(buf, sizeof buf, "(%a)", n->num);
      return buf;
    case Node::COMP:
      return "i2d(u[" + std::to_string(n->index) + "])";
    case Node::GD:
      return "g[" + std::to_string(n->index) + "]";
    case Node::NEG:
      return "(-" + code(n->a.get()) + ")";
    default:
      return "(" + code(n->a.get()) + " " + n->op + " " + code(n->b.get()) + ")";
  }
}

// counts of one side ("@" or terms [k*]name joined by '+'); false on error
bool side(const std::string &text, const std::vector<std::string> &comps, std::vector<int> &cnt,
          std::string &err) {
  size_t b = text.find_first_not_of(" \t\n");
  size_t e = text.find_last_not_of(" \t\n");
  if (b == std::string::npos) {
    err = "empty side";
    return false;
  }
  const std::string t = text.substr(b, e - b + 1);
  if (t == "@") return true;
  size_t pos = 0;
  while (pos <= t.size()) {
    size_t plus = t.find('+', pos);
    if (plus == std::string::npos) plus = t.size();
    std::string term = t.substr(pos, plus - pos);
    const size_t tb = term.find_first_not_of(" \t"), te = term.find_last_not_of(" \t");
    term = tb == std::string::npos ? "" : term.substr(tb, te - tb + 1);
    int k = 1;
    const size_t star = term.find('*');
    if (star != std::string::npos) {
      const std::string num = term.substr(0, star);
      char *endp = nullptr;
      const long v = std::strtol(num.c_str(), &endp, 10);
      bool digits = !num.empty();
      for (char ch : num)
        if (!std::isdigit((unsigned char)ch) && !std::isspace((unsigned char)ch)) digits = false;
      if (!digits || v < 1 || v > 1000000) {
        err = "bad multiplier in '" + term + "'";
        return false;
      }
      k = (int)v;
      term = term.substr(star + 1);
      const size_t nb = term.find_first_not_of(" \t");
      term = nb == std::string::npos ? "" : term.substr(nb);
    }
    int idx = -1;
    for (size_t p = 0; p < comps.size(); ++p)
      if (comps[p] == term) idx = (int)p;
    if (idx < 0) {
      err = "unknown compartment '" + term + "'";
      return false;
    }
    cnt[idx] += k;
    pos = plus + 1;
  }
  return true;
}

}  // namespace

int mparse(const char *const *transitions, int n_trans, const char *const *compartments,
           int n_comp, const char *const *gdata_names, int n_gdata, ParsedModel &out,
           std::string &err) {
  if (n_trans < 1 || n_trans > SG_MAX_TRANS || n_comp < 1 || n_comp > SG_MAX_COMP ||
      n_gdata < 0 || n_gdata > SG_MAX_GDATA || !transitions || !compartments ||
      (n_gdata > 0 && !gdata_names)) {
    err = "sizes out of range";
    return SG_ERR_ARG;
  }
  std::vector<std::string> comps, gn;
  for (int p = 0; p < n_comp; ++p) {
    if (!compartments[p]) return SG_ERR_ARG;
    comps.emplace_back(compartments[p]);
  }
  for (int q = 0; q < n_gdata; ++q) {
    if (!gdata_names[q]) return SG_ERR_ARG;
    gn.emplace_back(gdata_names[q]);
  }
  std::vector<std::string> all(comps);
  all.insert(all.end(), gn.begin(), gn.end());
  for (size_t i = 0; i < all.size(); ++i) {
    bool ok = !all[i].empty() && name_start(all[i][0]);
    for (char ch : all[i]) ok = ok && name_char(ch);
    for (size_t j = 0; j < i; ++j) ok = ok && all[j] != all[i];
    if (!ok) {
      err = "compartment and gdata names must be distinct identifiers ('" + all[i] + "')";
      return SG_ERR_PARSE;
    }
  }
  out.C = n_comp;
  out.T = n_trans;
  out.S.assign((size_t)n_comp * n_trans, 0);
  out.G.assign((size_t)n_trans * n_trans, 0);
  out.rate_code.clear();
  std::vector<std::vector<char>> rd;
  for (int j = 0; j < n_trans; ++j) {
    if (!transitions[j]) return SG_ERR_ARG;
    const std::string t(transitions[j]);
    const size_t a1 = t.find("->");
    const size_t a2 = a1 == std::string::npos ? a1 : t.find("->", a1 + 2);
    if (a1 == std::string::npos || a2 == std::string::npos ||
        t.find("->", a2 + 2) != std::string::npos) {
      err = "transition " + std::to_string(j) + ": expected 'LHS -> propensity -> RHS'";
      return SG_ERR_PARSE;
    }
    std::vector<int> lhs(n_comp, 0), rhs(n_comp, 0);
    std::string e;
    if (!side(t.substr(0, a1), comps, lhs, e) || !side(t.substr(a2 + 2), comps, rhs, e)) {
      err = "transition " + std::to_string(j) + ": " + e;
      return SG_ERR_PARSE;
    }
    for (int p = 0; p < n_comp; ++p) {
      const int d = rhs[p] - lhs[p];
      if (d < -127 || d > 127) {
        err = "transition " + std::to_string(j) + ": change out of range";
        return SG_ERR_PARSE;
      }
      out.S[(size_t)j * n_comp + p] = d;
    }
    const std::string prop = t.substr(a1 + 2, a2 - a1 - 2);
    Parser ps(prop.c_str(), comps, gn);
    std::unique_ptr<Node> tree = ps.parse(e);
    if (!tree) {
      err = "transition " + std::to_string(j) + ": " + e;
      return SG_ERR_PARSE;
    }
    std::vector<char> r(n_comp, 0);
    reads(tree.get(), r);
    rd.push_back(r);
    out.rate_code.push_back(code(tree.get()));
  }
  // G[k, j] = 1 when propensity k reads a compartment transition j changes
  for (int j = 0; j < n_trans; ++j)
    for (int k = 0; k < n_trans; ++k)
      for (int p = 0; p < n_comp; ++p)
        if (rd[k][p] && out.S[(size_t)j * n_comp + p] != 0) out.G[(size_t)j * n_trans + k] = 1;
  return SG_OK;
}

// ---------------------------------------------------------------------------
// Run-time compilation (NVRTC, loaded on first use so that the library loads
// on machines without it) and loading (CUDA runtime library API).
// ---------------------------------------------------------------------------
namespace {

#include "sg_jit_sources.inc"  // kJitNames / kJitSources: the kernel headers

struct Nvrtc {
  bool ok = false;
  decltype(&nvrtcCreateProgram) create;
  decltype(&nvrtcAddNameExpression) add_name;
  decltype(&nvrtcCompileProgram) compile;
  decltype(&nvrtcGetProgramLogSize) log_size;
  decltype(&nvrtcGetProgramLog) log;
  decltype(&nvrtcGetCUBINSize) cubin_size;
  decltype(&nvrtcGetCUBIN) cubin;
  decltype(&nvrtcGetLoweredName) lowered;
  decltype(&nvrtcDestroyProgram) destroy;
};

const Nvrtc &nvrtc() {
  static Nvrtc n;
  static std::once_flag once;
  std::call_once(once, [] {
    void *h = nullptr;
    for (const char *name : {"libnvrtc.so.13", "libnvrtc.so"}) {
      h = dlopen(name, RTLD_NOW | RTLD_LOCAL);
      if (h) break;
    }
    if (!h) return;
    n.create = (decltype(n.create))dlsym(h, "nvrtcCreateProgram");
    n.add_name = (decltype(n.add_name))dlsym(h, "nvrtcAddNameExpression");
    n.compile = (decltype(n.compile))dlsym(h, "nvrtcCompileProgram");
    n.log_size = (decltype(n.log_size))dlsym(h, "nvrtcGetProgramLogSize");
    n.log = (decltype(n.log))dlsym(h, "nvrtcGetProgramLog");
    n.cubin_size = (decltype(n.cubin_size))dlsym(h, "nvrtcGetCUBINSize");
    n.cubin = (decltype(n.cubin))dlsym(h, "nvrtcGetCUBIN");
    n.lowered = (decltype(n.lowered))dlsym(h, "nvrtcGetLoweredName");
    n.destroy = (decltype(n.destroy))dlsym(h, "nvrtcDestroyProgram");
    n.ok = n.create && n.add_name && n.compile && n.log_size && n.log && n.cubin_size &&
           n.cubin && n.lowered && n.destroy;
  });
  return n;
}

}  // namespace

std::string generic_source(const ParsedModel &pm) {
  std::string s;
  s += "#include \"sg_common.h\"\n#include \"sg_device.cuh\"\nnamespace sg {\n";
  s += "template <> struct ModelTraits<SG_GENERIC> {\n";
  s += "  static constexpr int C = " + std::to_string(pm.C) + ", T = " + std::to_string(pm.T) +
       ", NV = 0, NK = 1;\n";
  s += "  __device__ static __forceinline__ void prepare(const double *, const double *, "
       "double *) {}\n";
  s += "  __device__ static __forceinline__ double rate_k(int j, const int *u, const double *, "
       "const double *g) {\n    switch (j) {\n";
  for (int j = 0; j < pm.T; ++j)
    s += "      case " + std::to_string(j) + ": return " + pm.rate_code[j] + ";\n";
  s += "    }\n    return 0.0;\n  }\n";
  s += "  __device__ static __forceinline__ double rate(int j, const int *u, const double *, "
       "const double *g) {\n    return rate_k(j, u, nullptr, g);\n  }\n};\n}  // namespace sg\n";
  s += "#include \"sg_kernels.cuh\"\n";
  return s;
}

int jit_build(const ParsedModel &pm, JitKernels &out, std::string &err) {
  const Nvrtc &n = nvrtc();
  if (!n.ok) {
    err = "NVRTC (libnvrtc.so.13) is not available";
    return SG_ERR_JIT;
  }
  const std::string src = generic_source(pm);
  nvrtcProgram prog;
  const int nh = (int)(sizeof kJitNames / sizeof kJitNames[0]);
  if (n.create(&prog, src.c_str(), "sg_generic.cu", nh, kJitSources, kJitNames) !=
      NVRTC_SUCCESS) {
    err = "nvrtcCreateProgram failed";
    return SG_ERR_JIT;
  }
  const std::string C = std::to_string(pm.C);
  const std::string names[JitKernels::kCount] = {
      "sg::k_days<" + std::to_string((int)SG_GENERIC) + ", false>",
      "sg::k_days<" + std::to_string((int)SG_GENERIC) + ", true>",
      "sg::k_events_e2<" + std::to_string((int)SG_GENERIC) + ", false>",
      "sg::k_events_e2<" + std::to_string((int)SG_GENERIC) + ", true>",
      "sg::k_record0<" + C + ", 0>"};
  for (const std::string &nm : names) n.add_name(prog, nm.c_str());
  // -default-device: the public header's entry-point declarations (host
  // functions, never called here) are read as device declarations
  const char *opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "-fmad=false",
                        "-default-device"};
  const nvrtcResult cr = n.compile(prog, (int)(sizeof opts / sizeof opts[0]), opts);
  if (cr != NVRTC_SUCCESS) {
    size_t ls = 0;
    n.log_size(prog, &ls);
    std::string log(ls, '\0');
    if (ls) n.log(prog, &log[0]);
    err = "NVRTC compile failed: " + log.substr(0, 4000);
    n.destroy(&prog);
    return SG_ERR_JIT;
  }
  size_t bytes = 0;
  n.cubin_size(prog, &bytes);
  std::vector<char> cubin(bytes);
  n.cubin(prog, cubin.data());
  std::string lowered[JitKernels::kCount];
  for (int i = 0; i < JitKernels::kCount; ++i) {
    const char *ln = nullptr;
    if (n.lowered(prog, names[i].c_str(), &ln) != NVRTC_SUCCESS || !ln) {
      err = "no lowered name for " + names[i];
      n.destroy(&prog);
      return SG_ERR_JIT;
    }
    lowered[i] = ln;
  }
  n.destroy(&prog);
  if (cudaFree(nullptr) != cudaSuccess ||
      cudaLibraryLoadData(&out.lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0) !=
          cudaSuccess) {
    cudaGetLastError();
    err = "loading the compiled kernels failed";
    return SG_ERR_JIT;
  }
  for (int i = 0; i < JitKernels::kCount; ++i) {
    if (cudaLibraryGetKernel(&out.k[i], out.lib, lowered[i].c_str()) != cudaSuccess) {
      cudaGetLastError();
      cudaLibraryUnload(out.lib);
      out.lib = nullptr;
      err = "kernel " + names[i] + " not found";
      return SG_ERR_JIT;
    }
  }
  cudaGetDevice(&out.device);
  return SG_OK;
}

void jit_release(JitKernels &k) {
  if (k.lib) cudaLibraryUnload(k.lib);
  k.lib = nullptr;
}

}  // namespace sg
