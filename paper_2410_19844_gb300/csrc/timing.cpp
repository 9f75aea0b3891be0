// Launch counting, optional per-kernel CUDA-event timing, and per-device
// one-time kernel set-up.
//
// Every launcher in this library constructs a KernelScope.  It always counts
// the launch; when timing is enabled it also records a CUDA event before and
// after the kernel on the launching stream, so the elapsed time of each
// launch is measured on the device, in stream order.  Timing is meant for
// uncaptured streams (enable it outside CUDA-graph capture).
#include <atomic>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "internal.h"

namespace sos {

namespace {

struct Rec {
    const char* name;
    cudaEvent_t start, stop;
};

std::atomic<int64_t> g_launches{0};
std::atomic<bool> g_timing{false};
std::mutex g_mu;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t take_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

std::mutex g_dev_mu;
std::map<std::pair<const void*, int>, int> g_dev_values;

}  // namespace

int per_device_value(const void* key, int* value, const std::function<int(int*)>& setup) {
    int dev = -1;
    SOS_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_dev_mu);
    auto it = g_dev_values.find({key, dev});
    if (it != g_dev_values.end()) {
        *value = it->second;
        return SOS_OK;
    }
    int v = 0;
    SOS_CHECK(setup(&v));
    g_dev_values[{key, dev}] = v;
    *value = v;
    return SOS_OK;
}

KernelScope::KernelScope(const char* name, cudaStream_t st) : name_(name), st_(st) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (!g_timing.load(std::memory_order_relaxed)) return;
    std::lock_guard<std::mutex> lock(g_mu);
    start_ = take_event();
    if (start_) cudaEventRecord(start_, st_);
}

KernelScope::~KernelScope() {
    if (!start_) return;
    std::lock_guard<std::mutex> lock(g_mu);
    cudaEvent_t stop = take_event();
    if (!stop) return;
    cudaEventRecord(stop, st_);
    g_recs.push_back({name_, start_, stop});
}

}  // namespace sos

using namespace sos;

extern "C" {

int64_t sos_launch_count(void) { return g_launches.load(); }

int sos_timing_enable(int on) {
    g_timing.store(on != 0);
    return SOS_OK;
}

int sos_timing_reset(void) {
    std::lock_guard<std::mutex> lock(g_mu);
    for (auto& r : g_recs) {
        cudaEventSynchronize(r.stop);
        g_pool.push_back(r.start);
        g_pool.push_back(r.stop);
    }
    g_recs.clear();
    return SOS_OK;
}

int sos_timing_report(char* buf, size_t cap) {
    if (!buf || cap == 0) return fail(SOS_E_INVALID, "sos_timing_report: bad buffer");
    std::lock_guard<std::mutex> lock(g_mu);
    std::map<std::string, std::pair<int64_t, double>> agg;
    for (auto& r : g_recs) {
        if (cudaEventSynchronize(r.stop) != cudaSuccess) return fail(SOS_E_CUDA, "sos_timing_report: event");
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.start, r.stop) != cudaSuccess)
            return fail(SOS_E_CUDA, "sos_timing_report: elapsed time");
        auto& a = agg[r.name];
        a.first += 1;
        a.second += ms;
    }
    std::string out;
    for (auto& kv : agg) {
        char line[256];
        std::snprintf(line, sizeof(line), "%s %lld %.6f\n", kv.first.c_str(), (long long)kv.second.first,
                      kv.second.second);
        out += line;
    }
    if (out.size() + 1 > cap) return fail(SOS_E_INVALID, "sos_timing_report: buffer too small");
    std::memcpy(buf, out.c_str(), out.size() + 1);
    return SOS_OK;
}

}  // extern "C"
