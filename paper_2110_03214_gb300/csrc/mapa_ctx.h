// Context object behind the opaque mapa_ctx handle (shared by the C ABI in
// mapa_capi.cpp and the serving loop in mapa_serve.cpp).  Not public.
#pragma once

#include <string>
#include <vector>

#include "mapa_internal.h"

namespace mapa {

struct TopoEntry {
    TopoDevice dev;
    std::vector<int32_t> wm;  // host copy of the n x n link weights (fill applied), for the simulator's logger
    bool live = false;
};

struct PatternEntry {
    PatternArgs args;
    uint64_t aut_order = 0;
};

}  // namespace mapa

struct mapa_ctx_s {
    mapa::Engine *engine = nullptr;
    int device = 0;
    std::string last_error;
    std::vector<mapa::TopoEntry> topos;
    std::vector<mapa::PatternEntry> patterns;
    std::vector<mapa::PatternArgs> pattern_args;  // contiguous copy handed to the engine
};
