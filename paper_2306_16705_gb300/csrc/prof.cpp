// Tracing: per-kernel-family launch counts and, when enabled, CUDA-event
// timing of every launch (nnqs_profile_*).  Events are recorded on the
// launching stream, so a family's time is the device time of its launches.
#include <cuda_runtime.h>

#include <atomic>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"

namespace nnqs {
namespace {

struct Family {
    std::string name;
    uint64_t launches = 0;
    double total_ms = 0.0;
    double flops = 0.0, bytes = 0.0;  // algorithmic work attributed by the launch sites
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
};

std::mutex g_mu;
std::vector<Family> g_fam;
std::atomic<uint64_t> g_launches{0};
std::atomic<bool> g_enabled{false};

int family_slot(const char *name) {
    for (size_t i = 0; i < g_fam.size(); ++i)
        if (g_fam[i].name == name) return (int)i;
    g_fam.push_back(Family{name});
    return (int)g_fam.size() - 1;
}

void drain_locked() {
    for (auto &f : g_fam) {
        for (auto &p : f.pending) {
            float ms = 0.f;
            if (cudaEventSynchronize(p.second) == cudaSuccess && cudaEventElapsedTime(&ms, p.first, p.second) == cudaSuccess)
                f.total_ms += ms;
            cudaEventDestroy(p.first);
            cudaEventDestroy(p.second);
        }
        f.pending.clear();
    }
}

}  // namespace

void note_work(const char *name, double flops, double bytes) {
    std::lock_guard<std::mutex> lk(g_mu);
    const int slot = family_slot(name);
    g_fam[slot].flops += flops;
    g_fam[slot].bytes += bytes;
}

cudaError_t note_launch() {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

void note_replay(uint64_t launches) { g_launches.fetch_add(launches, std::memory_order_relaxed); }

bool profiling_on() { return g_enabled.load(std::memory_order_relaxed); }

ProfScope::ProfScope(const char *name, cudaStream_t s) : name_(name), s_(s) {
    if (!g_enabled.load(std::memory_order_relaxed)) return;
    if (cudaEventCreate(&e0_) != cudaSuccess) return;
    if (cudaEventCreate(&e1_) != cudaSuccess) {
        cudaEventDestroy(e0_);
        return;
    }
    cudaEventRecord(e0_, s_);
    on_ = true;
}

ProfScope::~ProfScope() {
    std::lock_guard<std::mutex> lk(g_mu);
    const int slot = family_slot(name_);
    g_fam[slot].launches++;
    if (!on_) return;
    cudaEventRecord(e1_, s_);
    g_fam[slot].pending.push_back({e0_, e1_});
}

}  // namespace nnqs

extern "C" {

void nnqs_profile_enable(int on) { nnqs::g_enabled.store(on != 0); }

void nnqs_profile_reset(void) {
    std::lock_guard<std::mutex> lk(nnqs::g_mu);
    nnqs::drain_locked();
    for (auto &f : nnqs::g_fam) {
        f.launches = 0;
        f.total_ms = 0.0;
        f.flops = f.bytes = 0.0;
    }
}

int nnqs_profile_read(int index, char *name, int name_cap, uint64_t *launches, double *total_ms) {
    std::lock_guard<std::mutex> lk(nnqs::g_mu);
    nnqs::drain_locked();
    const int n = (int)nnqs::g_fam.size();
    if (index >= 0 && index < n) {
        const auto &f = nnqs::g_fam[index];
        if (name && name_cap > 0) {
            std::strncpy(name, f.name.c_str(), (size_t)name_cap - 1);
            name[name_cap - 1] = 0;
        }
        if (launches) *launches = f.launches;
        if (total_ms) *total_ms = f.total_ms;
    }
    return n;
}

int nnqs_profile_work(int index, double *flops, double *bytes) {
    std::lock_guard<std::mutex> lk(nnqs::g_mu);
    const int n = (int)nnqs::g_fam.size();
    if (index >= 0 && index < n) {
        if (flops) *flops = nnqs::g_fam[index].flops;
        if (bytes) *bytes = nnqs::g_fam[index].bytes;
    }
    return n;
}

uint64_t nnqs_launch_count(void) { return nnqs::g_launches.load(); }

}  // extern "C"
