// gc_tune.cu -- the batched form's tuning cache.
//
// The tuner (paper_1608_05138_gb300/tune.py) times the bitmatrix kernels of
// every size class under each block size, and the cut between the bitmatrix
// kernels and the general passes, on a held-out sample of graphs, and writes
// the best settings to a JSON file keyed by GPU name and graph class (the
// vertex-count bin of a size class):
//
//   { "NVIDIA GB300": { "small_n_max": 1024, "use_graph": 1,
//                       "block": { "64": 128, "128": 128, "256": 256,
//                                  "512": 256, "1024": 512 } } }
//
// gc_batch_create reads it (the file named by the environment variable
// GC_TUNE_CACHE, else tune_cache.json beside libgc.so); keys it does not
// know are ignored, and a missing file or GPU leaves the defaults.
#include <cuda_runtime.h>
#include <dlfcn.h>

#include <cctype>
#include <cstdlib>
#include <fstream>
#include <map>
#include <memory>
#include <sstream>
#include <string>

#include "gc_internal.h"

namespace gc {
namespace {

// A JSON value: only what the cache needs (objects, numbers, strings; arrays,
// booleans and null are parsed and ignored).
struct JValue {
  enum Kind { kNull, kNumber, kString, kObject, kOther } kind = kNull;
  double num = 0;
  std::string str;
  std::map<std::string, std::unique_ptr<JValue>> obj;
};

class JParser {
 public:
  explicit JParser(const std::string& t) : t_(t) {}
  bool parse(JValue* v) {
    if (!value(v, 0)) return false;
    ws();
    return i_ == t_.size();
  }

 private:
  const std::string& t_;
  size_t i_ = 0;
  void ws() {
    while (i_ < t_.size() && std::isspace((unsigned char)t_[i_])) ++i_;
  }
  bool lit(const char* w) {
    const size_t n = std::char_traits<char>::length(w);
    if (t_.compare(i_, n, w) != 0) return false;
    i_ += n;
    return true;
  }
  bool string(std::string* out) {
    if (i_ >= t_.size() || t_[i_] != '"') return false;
    ++i_;
    while (i_ < t_.size() && t_[i_] != '"') {
      if (t_[i_] == '\\') {
        if (++i_ >= t_.size()) return false;
        const char c = t_[i_];
        out->push_back(c == 'n' ? '\n' : c == 't' ? '\t' : c);  // \uXXXX is not needed here
      } else {
        out->push_back(t_[i_]);
      }
      ++i_;
    }
    if (i_ >= t_.size()) return false;
    ++i_;
    return true;
  }
  bool value(JValue* v, int depth) {
    if (depth > 32) return false;
    ws();
    if (i_ >= t_.size()) return false;
    const char c = t_[i_];
    if (c == '{') {
      ++i_;
      v->kind = JValue::kObject;
      ws();
      if (i_ < t_.size() && t_[i_] == '}') {
        ++i_;
        return true;
      }
      for (;;) {
        ws();
        std::string key;
        if (!string(&key)) return false;
        ws();
        if (i_ >= t_.size() || t_[i_] != ':') return false;
        ++i_;
        auto child = std::make_unique<JValue>();
        if (!value(child.get(), depth + 1)) return false;
        v->obj[key] = std::move(child);
        ws();
        if (i_ < t_.size() && t_[i_] == ',') {
          ++i_;
          continue;
        }
        if (i_ < t_.size() && t_[i_] == '}') {
          ++i_;
          return true;
        }
        return false;
      }
    }
    if (c == '[') {
      ++i_;
      v->kind = JValue::kOther;
      ws();
      if (i_ < t_.size() && t_[i_] == ']') {
        ++i_;
        return true;
      }
      for (;;) {
        JValue skip;
        if (!value(&skip, depth + 1)) return false;
        ws();
        if (i_ < t_.size() && t_[i_] == ',') {
          ++i_;
          continue;
        }
        if (i_ < t_.size() && t_[i_] == ']') {
          ++i_;
          return true;
        }
        return false;
      }
    }
    if (c == '"') {
      v->kind = JValue::kString;
      return string(&v->str);
    }
    if (lit("true") || lit("false") || lit("null")) {
      v->kind = JValue::kOther;
      return true;
    }
    const char* b = t_.c_str() + i_;
    char* e = nullptr;
    v->num = std::strtod(b, &e);
    if (e == b) return false;
    v->kind = JValue::kNumber;
    i_ += (size_t)(e - b);
    return true;
  }
};

const JValue* member(const JValue* v, const std::string& k) {
  if (!v || v->kind != JValue::kObject) return nullptr;
  auto it = v->obj.find(k);
  return it == v->obj.end() ? nullptr : it->second.get();
}

std::string cache_path() {
  if (const char* e = getenv("GC_TUNE_CACHE")) return e;
  Dl_info info;
  if (dladdr((void*)&cache_path, &info) && info.dli_fname) {
    std::string so = info.dli_fname;
    const size_t slash = so.find_last_of('/');
    return (slash == std::string::npos ? std::string(".") : so.substr(0, slash)) + "/tune_cache.json";
  }
  return "tune_cache.json";
}

}  // namespace

bool load_tuned_config(BatchConfig* cfg, std::string* source) {
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  const std::string path = cache_path();
  std::ifstream f(path);
  if (!f) return false;
  std::stringstream ss;
  ss << f.rdbuf();
  const std::string text = ss.str();
  JValue root;
  if (!JParser(text).parse(&root)) return false;
  const JValue* gpu = member(&root, prop.name);
  if (!gpu) return false;
  BatchConfig c = *cfg;
  if (const JValue* v = member(gpu, "small_n_max"))
    if (v->kind == JValue::kNumber && v->num >= 0 && v->num <= kSmallClassN[kSmallClasses - 1])
      c.small_n_max = (int32_t)v->num;
  if (const JValue* v = member(gpu, "use_graph"))
    if (v->kind == JValue::kNumber) c.use_graph = v->num != 0;
  if (const JValue* v = member(gpu, "max_inflight"))
    if (v->kind == JValue::kNumber && v->num >= 1 && v->num <= kMaxInflight) c.max_inflight = (int32_t)v->num;
  if (const JValue* blk = member(gpu, "block"))
    for (int k = 0; k < kSmallClasses; ++k)
      if (const JValue* v = member(blk, std::to_string(kSmallClassN[k])))
        if (v->kind == JValue::kNumber) {
          const int b = (int)v->num;
          if (b == 64 || b == 128 || b == 256 || b == 512) c.class_block[k] = b;
        }
  *cfg = c;
  if (source) *source = path + " [" + prop.name + "]";
  return true;
}

}  // namespace gc
