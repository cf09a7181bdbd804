#pragma once
#include "controller.cuh"
#include "pch_common.cuh"

namespace pch {

struct SrcDev {
    int inst, kind, vertex, face;
    int label;              // index of the source in the caller's list (Voronoi labels)
    int pad;
    double bary[3];
};

struct SolveCfg {
    int control;
    int loop;
    long long k;
    long long max_iters;
    int prop_threads;
    int prop_blocks_per_sm;
    int key_bits;
    int trim;
    int edge_sort;          // sort new windows by (instance, half-edge) instead of by instance
    int unroll;
    int full_fan;
    int profile;
    int hops;
    int tail_cut;           // stop chaining once the selected list is dry and fewer entries are queued
    int take_min;           // fresh windows a propagation warp may take at once, at least (32: a full warp)
    int stride_T;           // PCH_CONTROL_STRIDED: virtual threads of the strided selection (else 0)
    int stride_m;           // PCH_CONTROL_STRIDED: windows each of them selects (1, 2, 4, 8 or 16)
    int prov;               // record distance events for geodesic paths
    const float* mlp;
};

enum { kOutHost = 0, kOutDevice = 1, kOutNone = 2 };

long long default_k();
int default_hops();
int default_prop_blocks_per_sm(int block);
int default_tail_cut();
int default_take_min();
const float* mlp_device_params();

// prov: also record every distance event that lowered a vertex's distance (geodesic
// paths); the records stay in the workspace after the call.
pch_status solve_instances(pch_mesh* const* meshes, int n_inst, const SrcDev* srcs, int n_src,
                           const pch_options* opt, double* const* outs, int out_mode, pch_stats* stats,
                           int prov = 0);

}  // namespace pch
