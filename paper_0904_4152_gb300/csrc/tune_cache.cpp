// Persisted launch shapes (the runtime configuration file of Sec. 3: measured per-machine choices
// kept in a file that later runs read).  A text file named by HN_TUNE_CACHE holds one line per
// (GPU name, level, precision, solver, coarse solver, coarse level):
//
//   <gpu name>|<L>|<prec>|<solver>|<coarse solver>|<coarse L> <tail_level> <cluster> <pdl> <staged> <dsm> <fuse_up> <mid> <sweep>
//
// (an entry without the last field has sweep 0)
// hn_mg_autotune stores its result there; hn_mg_setup applies a stored shape to a new hierarchy
// of the same key.  Host code only: no device call.
#include <cstdio>
#include <cstring>
#include <fstream>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>
#include <unistd.h>

#include "engine.h"
#include "../../include/hn_tune.h"

namespace {

std::mutex g_file_mu;   // one writer at a time within the process

std::string make_key(const char* gpu, int L, int prec, int solver, int coarse_solver, int coarse_L) {
  std::string g(gpu ? gpu : "");
  for (char& c : g)
    if (c == '|' || c == '\n' || c == '\r') c = '_';
  std::ostringstream os;
  os << g << '|' << L << '|' << prec << '|' << solver << '|' << coarse_solver << '|' << coarse_L;
  return os.str();
}

// the key of a line (everything up to the last '|' field and the following space), or "" for a
// line that is not an entry
bool split_line(const std::string& line, std::string& key, std::string& rest) {
  size_t bar = line.rfind('|');
  if (bar == std::string::npos) return false;
  size_t sp = line.find(' ', bar);
  if (sp == std::string::npos) return false;
  key = line.substr(0, sp);
  rest = line.substr(sp + 1);
  return true;
}

bool parse_shape(const std::string& rest, hn_tuning* t) {
  std::istringstream is(rest);
  hn_tuning v{};
  if (!(is >> v.tail_level >> v.cluster >> v.pdl >> v.staged >> v.dsm >> v.fuse_up >> v.mid)) return false;
  if (!(is >> v.sweep)) {
    if (!is.eof()) return false;                  // a seventh field that is not a number
    v.sweep = 0;
  }
  std::string extra;
  if (is >> extra) return false;
  const int c = v.cluster;
  if (v.tail_level < HN_MIN_LEVEL || v.tail_level > HN_MAX_LEVEL || !(c == 1 || c == 2 || c == 4 || c == 8 || c == 16) ||
      v.pdl < 0 || v.pdl > 3 || (v.staged != 0 && v.staged != 1) || (v.dsm != 0 && v.dsm != 1) ||
      (v.fuse_up != 0 && v.fuse_up != 1) || v.mid < 0 || v.mid > HN_MAX_LEVEL || v.sweep < 0 || v.sweep > 2)
    return false;
  *t = v;
  return true;
}

}  // namespace

extern "C" {

hn_status hn_tune_cache_lookup(const char* path, const char* gpu, int L, int prec, int solver,
                               int coarse_solver, int coarse_L, hn_tuning* out) {
  hn::clear_error();
  if (!path || !gpu || !out) return hn::set_error(HN_ERR_ARG, "null argument");
  std::lock_guard<std::mutex> lk(g_file_mu);
  std::ifstream f(path);
  if (!f) return hn::set_error(HN_ERR_STATE, "no launch-shape file %s", path);
  const std::string want = make_key(gpu, L, prec, solver, coarse_solver, coarse_L);
  std::string line, key, rest;
  bool found = false;
  while (std::getline(f, line)) {
    if (!split_line(line, key, rest) || key != want) continue;
    hn_tuning t;
    if (parse_shape(rest, &t)) { *out = t; found = true; }   // the last valid entry wins
  }
  return found ? HN_OK : hn::set_error(HN_ERR_STATE, "no launch shape stored for %s", want.c_str());
}

hn_status hn_tune_cache_store(const char* path, const char* gpu, int L, int prec, int solver,
                              int coarse_solver, int coarse_L, const hn_tuning* t) {
  hn::clear_error();
  if (!path || !gpu || !t) return hn::set_error(HN_ERR_ARG, "null argument");
  std::string probe;
  {
    std::ostringstream os;
    os << t->tail_level << ' ' << t->cluster << ' ' << t->pdl << ' ' << t->staged << ' ' << t->dsm << ' '
       << t->fuse_up << ' ' << t->mid << ' ' << t->sweep;
    probe = os.str();
  }
  hn_tuning check;
  if (!parse_shape(probe, &check)) return hn::set_error(HN_ERR_ARG, "launch shape out of range");
  std::lock_guard<std::mutex> lk(g_file_mu);
  const std::string want = make_key(gpu, L, prec, solver, coarse_solver, coarse_L);
  std::vector<std::string> lines;
  {
    std::ifstream f(path);
    std::string line, key, rest;
    while (f && std::getline(f, line)) {
      if (split_line(line, key, rest) && key == want) continue;   // replaced below
      lines.push_back(line);
    }
  }
  lines.push_back(want + ' ' + probe);
  // write a new file next to the old one and rename it over: a reader sees the old or the new
  // file, never a partial one
  const std::string tmp = std::string(path) + ".tmp." + std::to_string((long long)getpid());
  {
    std::ofstream o(tmp, std::ios::trunc);
    if (!o) return hn::set_error(HN_ERR_STATE, "cannot write %s", tmp.c_str());
    for (const std::string& l : lines) o << l << '\n';
    if (!o.flush()) { std::remove(tmp.c_str()); return hn::set_error(HN_ERR_STATE, "cannot write %s", tmp.c_str()); }
  }
  if (std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    return hn::set_error(HN_ERR_STATE, "cannot replace %s", path);
  }
  return HN_OK;
}

}  // extern "C"
