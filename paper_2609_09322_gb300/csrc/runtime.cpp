// runtime.cpp -- environment settings and host-side fault injection.
//
// GBD_FAULT makes the N-th call at a named site fail on the host, e.g.
// GBD_FAULT=alloc:2 fails the second volume allocation with GBD_ERR_NOMEM.
// Faults are only ever injected on the host; no device work is disturbed.
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>

#include "runtime.h"

namespace gbd {
namespace {

std::mutex g_fault_mu;
int g_alloc_calls = 0, g_admit_calls = 0;

int parse_site(const char *spec, const char *site)
{
    if (!spec) return 0;
    const size_t len = std::strlen(site);
    for (const char *p = spec; p && *p;) {
        if (std::strncmp(p, site, len) == 0 && p[len] == ':') return std::atoi(p + len + 1);
        p = std::strchr(p, ',');
        if (p) ++p;
    }
    return 0;
}

}  // namespace

bool graphs_enabled()
{
    const char *s = std::getenv("GBD_GRAPHS");
    return !(s && s[0] == '0');
}

bool fault_injected(const char *site)
{
    const char *spec = std::getenv("GBD_FAULT");
    const int n = parse_site(spec, site);
    if (n <= 0) return false;
    std::lock_guard<std::mutex> lock(g_fault_mu);
    int &calls = std::strcmp(site, "alloc") == 0 ? g_alloc_calls : g_admit_calls;
    return ++calls == n;
}

void reset_fault_counters()
{
    std::lock_guard<std::mutex> lock(g_fault_mu);
    g_alloc_calls = g_admit_calls = 0;
}

}  // namespace gbd
