// Gauge handle and host-side batch builders shared by the launchers.
#pragma once

#include <vector>

#include "bpp_internal.h"

struct bpp_gauge_s {
    bpp::Geom g;
    int64_t V = 0, Vh = 0, stride = 0;
    int device = 0;
    void* links[bpp::NPREC] = {};    // per storage format: 8 link fields [parity][mu]
    // every link is SU(3) (checked at creation): FP32 also keeps the two-row
    // form (rows 1 and 2; row 3 = conj(row1 x row2) is rebuilt)
    bool su3 = false;
    void* links12[bpp::NPREC] = {};  // FP32: 3 planes of float4
    bool has_clover = false;
    double clov_kappa = 0.0, clov_csw = 0.0;
    void* clover[bpp::NPREC] = {};   // per storage format: A_e, A_o, Ainv_e, Ainv_o
};

namespace bpp {

using Gauge = bpp_gauge_s;

inline size_t clover_alloc_bytes(int prec, int64_t stride) {
    return (size_t)stride * ((prec == P64 || prec == P64S) ? 576 : prec == P32 ? 288 : 144);
}

inline size_t link12_alloc_bytes(int prec, int64_t stride) { return (size_t)stride * (prec == P32 ? 48 : 0); }

inline LinkView link12_view(const Gauge& G, int prec, int parity, int mu) {
    LinkView v;
    v.data = static_cast<const char*>(G.links12[prec]) + (size_t)(parity * 4 + mu) * link12_alloc_bytes(prec, G.stride);
    v.stride = G.stride;
    return v;
}

inline LinkView link_view(const Gauge& G, int prec, int parity, int mu) {
    LinkView v;
    v.data = static_cast<const char*>(G.links[prec]) + (size_t)(parity * 4 + mu) * link_alloc_bytes(prec, G.stride);
    v.stride = G.stride;
    return v;
}

// which: 0 = A, 1 = A^-1
inline CloverView clover_view(const Gauge& G, int prec, int which, int parity) {
    CloverView v;
    v.stride = G.stride;
    v.data = G.has_clover ? static_cast<const char*>(G.clover[prec]) +
                                (size_t)(which * 2 + parity) * clover_alloc_bytes(prec, G.stride)
                          : nullptr;
    return v;
}

// Host description of a batch: one SysDesc per system plus the device copy.
struct Batch {
    int prec = P64;
    std::vector<SysDesc> sys;
    DevBuf dsys;
    size_t vec_bytes = 0;   // bytes of one batch vector (all systems, one parity)
    bool uniform = true;
    int Vh_max = 0;
    // FP32: the systems' links in the two-row form (set before the first
    // batch_add; every gauge added must then be SU(3))
    bool comp = false;
    void upload(cudaStream_t s) {
        dsys.alloc(sys.size() * sizeof(SysDesc), s);
        BPP_CUDA(cudaMemcpyAsync(dsys.p, sys.data(), sys.size() * sizeof(SysDesc), cudaMemcpyHostToDevice, s));
    }
    const SysDesc* dev() const { return dsys.as<SysDesc>(); }
    int nsys() const { return (int)sys.size(); }
    // half-lattice sites of all systems
    double sites() const {
        double n = 0;
        for (auto& d : sys) n += d.g.Vh;
        return n;
    }
};

// Appends one system on gauge G (kappa, clover if csw != 0) to batch b.
void batch_add(Batch& b, const Gauge& G, double kappa, bool clover);
// Whether hopping kernels on gauge G in precision prec may use the two-row
// links (G is SU(3), prec is FP32, and BPP_LINK_COMPRESSION is not 0).
bool link_compression(const Gauge& G, int prec);
// Grid and block map for a launch over all systems with `sites_per_block`.
BlockMap block_map(const Batch& b, int sites_per_block, int& nblocks);

}  // namespace bpp
