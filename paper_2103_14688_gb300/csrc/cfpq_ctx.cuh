// cfpq_ctx.cuh -- the context object behind cfpq_ctx* (internal).
#pragma once
#include <memory>
#include <string>
#include <vector>

#include "cfpq_engine.cuh"
#include "cfpq_paths_host.h"

struct cfpq_ctx {
    using Allocator = cfpq::Allocator;
    using GraphDev = cfpq::GraphDev;
    using QueryDev = cfpq::QueryDev;
    using Executor = cfpq::Executor;
    using DBuf = cfpq::DBuf;
    cfpq_options opt;
    cudaStream_t stream = nullptr;
    Allocator A;
    std::string err;
    GraphDev graph;
    bool has_graph = false;
    bool has_rsm = false;
    QueryDev query;
    Executor exec;
    uint64_t exec_generation = ~0ull;
    bool exec_dirty = true;
    bool has_result = false;
    uint64_t result_gen = 0;  // bumped whenever the result changes or is dropped
    // after a multiple-source run: per vertex 1 if it was a source (only those
    // rows of the result are exact); empty after a full run
    std::vector<uint8_t> result_sources;
    // resume: M2 to start the next runs from (cfpq_set_start), host layout
    // start_B x start_n rows of ceil(start_n / 64) words
    std::vector<uint64_t> start_bits;
    bool has_start = false;
    uint32_t start_B = 0, start_n = 0;
    // column sharding (cfpq_shard_*): this rank's output columns [c0, c1)
    bool shard_on = false;
    uint32_t shard_c0 = 0, shard_c1 = 0;
    DBuf shard_cnt;  // per box: new edges, new to this rank (k_shard_apply)
    // batch (its graphs' and queries' buffers come from bslab, declared
    // first so that it outlives them)
    cfpq::SlabArena bslab;
    std::vector<std::unique_ptr<GraphDev>> bgraphs;
    std::vector<std::unique_ptr<QueryDev>> bqueries;
    Executor bexec;
    bool has_batch = false;
    // scratch for small transfers
    DBuf counter;
    DBuf rows_ptrs, rows_idx, rows_out;
    // path extraction: backward layers on the device; the enumerator (host
    // copies and memo) of result result_gen
    cfpq::PathsDev paths;
    std::unique_ptr<cfpq::PathEnum<cfpq::HostRSM>> penum;
    uint64_t penum_gen = ~0ull;
    ~cfpq_ctx() {
        // Buffers are released by their destructors through A (declared first).
    }
};

