// cg_fault.h - host-side fault injection, for tests of the error paths that
// fault, trap or hang no GPU.
//
// A plan is "site:n[:ms]" entries separated by commas. The n-th time (from 1)
// a context or server reaches `site`, the library behaves as if that step had
// failed: an allocation ("alloc", CG_ENOMEM), an input copy ("h2d",
// CG_ECUDA), a bounded device wait ("timeout", CG_ETIMEOUT), a kernel's
// consistency check ("kernel", CG_EKERNEL), input validation ("bad_graph",
// CG_EGRAPH), server admission ("admit", CG_EBUSY), a server worker that
// stalls for ms milliseconds before its batch ("queue_stall"), or a server
// batch whose first device wait reports a timeout ("batch_timeout"). Plans come from
// the CG_FAULT environment variable when a context or server starts, or from
// cg_set_fault.
#pragma once

#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

namespace cg {

class FaultPlan {
 public:
  void set(const char* spec) {
    std::lock_guard<std::mutex> lk(mu_);
    entries_.clear();
    if (!spec) return;
    std::string s(spec);
    size_t i = 0;
    while (i < s.size()) {
      size_t j = s.find(',', i);
      if (j == std::string::npos) j = s.size();
      std::string item = s.substr(i, j - i);
      i = j + 1;
      size_t c1 = item.find(':');
      if (c1 == std::string::npos || c1 == 0) continue;
      Entry e;
      e.site = item.substr(0, c1);
      size_t c2 = item.find(':', c1 + 1);
      e.at = std::atoll(item.substr(c1 + 1, c2 == std::string::npos ? std::string::npos : c2 - c1 - 1).c_str());
      e.ms = c2 == std::string::npos ? 0 : std::atoi(item.substr(c2 + 1).c_str());
      if (e.at >= 1) entries_.push_back(e);
    }
  }
  void from_env() { set(std::getenv("CG_FAULT")); }
  // Counts one arrival at `site`; true when it is the planned one.
  bool hit(const char* site, int* ms = nullptr) {
    std::lock_guard<std::mutex> lk(mu_);
    for (Entry& e : entries_) {
      if (e.site != site) continue;
      if (++e.seen == e.at) {
        if (ms) *ms = e.ms;
        return true;
      }
    }
    return false;
  }

 private:
  struct Entry {
    std::string site;
    long long at = 0, seen = 0;
    int ms = 0;
  };
  std::mutex mu_;
  std::vector<Entry> entries_;
};

}  // namespace cg
