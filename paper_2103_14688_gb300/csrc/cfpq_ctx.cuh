// cfpq_ctx.cuh -- the context object behind cfpq_ctx* (internal).
#pragma once
#include <memory>
#include <string>
#include <vector>

#include "cfpq_engine.cuh"

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
    // batch
    std::vector<std::unique_ptr<GraphDev>> bgraphs;
    std::vector<std::unique_ptr<QueryDev>> bqueries;
    Executor bexec;
    bool has_batch = false;
    // scratch for small transfers
    DBuf counter;
    DBuf rows_ptrs, rows_idx, rows_out;
    ~cfpq_ctx() {
        // Buffers are released by their destructors through A (declared first).
    }
};

