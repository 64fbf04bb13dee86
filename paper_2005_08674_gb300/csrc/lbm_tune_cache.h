// lbm_tune_cache.h -- persistent record of the autotuners' choices (host
// code only, no CUDA): a small JSON file mapping a key -- device name, driver
// and runtime versions, the library's build id, the kind of tuning (single
// domain or batch), storage, collision model, storage-shift form and a size
// class -- to the launch shape that won, so that a later process with the
// same key applies it without timing the candidates again.
//
// File format (written by store(), read back by load()):
//   {"lbm_tune_cache": 1, "entries": [
//     {"key": "...", "name": value, ...},
//     ...]}
// with numeric values only.  Anything that does not parse as that format
// reads as an empty cache (the autotuner then times as usual and rewrites
// the file); a file that cannot be written is left alone.  Writes go to a
// temporary file that is renamed over the old one.
#pragma once

#include <cerrno>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

namespace lbmtune {

struct Entry {
  std::string key;
  std::vector<std::pair<std::string, double>> values;

  bool get(const char* name, double* out) const {
    for (const auto& v : values)
      if (v.first == name) {
        *out = v.second;
        return true;
      }
    return false;
  }
};

// Size class of an extent: ceil(log2(n)) (n >= 1), so 129..256 share a class.
inline int size_class(long long n) {
  int c = 0;
  while (c < 62 && (1LL << c) < n) ++c;
  return c;
}

// Key of one tuning problem.  `dims` are extents whose size classes enter
// the key (nx, ny for one domain; instance count and total nodes for a batch).
inline std::string make_key(const char* device, int driver, int runtime, const char* build, const char* kind,
                            int storage, int model, bool shift, const std::vector<long long>& dims) {
  std::string k;
  k += device ? device : "?";
  k += "|drv" + std::to_string(driver) + "|rt" + std::to_string(runtime);
  k += std::string("|build:") + (build ? build : "?");
  k += std::string("|") + kind;
  k += "|storage" + std::to_string(storage) + "|model" + std::to_string(model) + (shift ? "|shift" : "|plain");
  for (long long d : dims) k += "|c" + std::to_string(size_class(d));
  // a key is a JSON string: keep it to characters that need no escaping
  for (char& ch : k)
    if (ch == '"' || ch == '\\' || (unsigned char)ch < 0x20) ch = '_';
  return k;
}

namespace detail {
inline void skip_ws(const char*& p) {
  while (*p == ' ' || *p == '\n' || *p == '\r' || *p == '\t') ++p;
}
inline bool expect(const char*& p, char c) {
  skip_ws(p);
  if (*p != c) return false;
  ++p;
  return true;
}
inline bool parse_string(const char*& p, std::string& out) {
  skip_ws(p);
  if (*p != '"') return false;
  ++p;
  out.clear();
  while (*p && *p != '"') {
    if (*p == '\\' || (unsigned char)*p < 0x20) return false;  // never written
    out += *p++;
  }
  if (*p != '"') return false;
  ++p;
  return true;
}
inline bool parse_number(const char*& p, double& out) {
  skip_ws(p);
  errno = 0;
  char* end = nullptr;
  out = std::strtod(p, &end);
  if (end == p || errno != 0 || !std::isfinite(out)) return false;
  p = end;
  return true;
}
}  // namespace detail

// Parse the cache text; false (and no entries) if it is not in the format.
inline bool parse(const std::string& text, std::vector<Entry>& out) {
  using namespace detail;
  out.clear();
  const char* p = text.c_str();
  std::string name;
  double version = 0.0;
  if (!expect(p, '{') || !parse_string(p, name) || name != "lbm_tune_cache" || !expect(p, ':') ||
      !parse_number(p, version) || version != 1.0 || !expect(p, ',') || !parse_string(p, name) ||
      name != "entries" || !expect(p, ':') || !expect(p, '['))
    return false;
  skip_ws(p);
  if (*p == ']') {
    ++p;
  } else {
    for (;;) {
      Entry e;
      if (!expect(p, '{') || !parse_string(p, name) || name != "key" || !expect(p, ':') || !parse_string(p, e.key))
        return out.clear(), false;
      skip_ws(p);
      while (*p == ',') {
        ++p;
        double v = 0.0;
        if (!parse_string(p, name) || !expect(p, ':') || !parse_number(p, v)) return out.clear(), false;
        e.values.emplace_back(name, v);
        skip_ws(p);
      }
      if (!expect(p, '}')) return out.clear(), false;
      out.push_back(std::move(e));
      skip_ws(p);
      if (*p == ',') {
        ++p;
        continue;
      }
      if (!expect(p, ']')) return out.clear(), false;
      break;
    }
  }
  if (!expect(p, '}')) return out.clear(), false;
  skip_ws(p);
  return *p == '\0' ? true : (out.clear(), false);
}

inline std::string format(const std::vector<Entry>& entries) {
  std::string s = "{\"lbm_tune_cache\": 1, \"entries\": [";
  char num[64];
  for (size_t k = 0; k < entries.size(); ++k) {
    s += k ? ",\n  " : "\n  ";
    s += "{\"key\": \"" + entries[k].key + "\"";
    for (const auto& v : entries[k].values) {
      std::snprintf(num, sizeof num, "%.17g", v.second);
      s += ", \"" + v.first + "\": " + num;
    }
    s += "}";
  }
  s += "]}\n";
  return s;
}

// Entries of the file at `path`; empty if it is missing or not in the format.
inline std::vector<Entry> load(const std::string& path) {
  std::vector<Entry> out;
  FILE* f = std::fopen(path.c_str(), "rb");
  if (!f) return out;
  std::string text;
  char buf[4096];
  size_t n;
  while ((n = std::fread(buf, 1, sizeof buf, f)) > 0 && text.size() < (16u << 20)) text.append(buf, n);
  std::fclose(f);
  if (!parse(text, out)) out.clear();
  return out;
}

inline bool lookup(const std::string& path, const std::string& key, Entry* out) {
  for (auto& e : load(path))
    if (e.key == key) {
      *out = std::move(e);
      return true;
    }
  return false;
}

// Add or replace the entry with e.key; false if the file cannot be written.
inline bool store(const std::string& path, const Entry& e) {
  std::vector<Entry> entries = load(path);
  bool replaced = false;
  for (auto& x : entries)
    if (x.key == e.key) {
      x = e;
      replaced = true;
    }
  if (!replaced) entries.push_back(e);
  const std::string tmp = path + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "wb");
  if (!f) return false;
  const std::string text = format(entries);
  const bool ok = std::fwrite(text.data(), 1, text.size(), f) == text.size();
  if (std::fclose(f) != 0 || !ok) {
    std::remove(tmp.c_str());
    return false;
  }
  if (std::rename(tmp.c_str(), path.c_str()) != 0) {
    std::remove(tmp.c_str());
    return false;
  }
  return true;
}

}  // namespace lbmtune
