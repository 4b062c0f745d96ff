// model.cuh -- compiled models and ciphertext handles (layers.cu), shared with
// the serving loop (server.cu).
#pragma once
#include "ops.cuh"

// cached encoded plaintexts of a compiled model (nullptr: encode every call)
struct PtCache {
    std::map<std::string, DBuf> pts;
    // a convolution whose masks take more than this many bytes (0: no limit) keeps only their
    // sparse description here and encodes them at every run, output channels in groups
    // whose masks fit the budget
    size_t mask_budget = 0;
    std::map<std::string, std::vector<size_t>> desc;   // word offsets of off / pos / val, counts
};

struct LayerSpec {
    u32 op = 0, ci = 0, co = 0, k = 0, s = 1;
    std::vector<double> w, b;
};

struct Plan {
    u32 stride = 0, levels = 0, C = 1;   // C: input channels of the first convolution
    std::vector<int> steps;
};

struct ModelGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    Cts in, out;
    u64 kernels = 0;   // kernel nodes in the graph
};

// Handles share ownership of their context: it is torn down when the last
// context, ciphertext or model handle that refers to it has been freed.
struct he_model {
    std::shared_ptr<Ctx> keep;
    Ctx *c = nullptr;
    std::vector<LayerSpec> layers;
    u32 W_img = 0, H_img = 0, spc = 0;
    Plan plan;
    bool literal = false;                  // compiled under the paper-order schedule
    PtCache pc;
    bool pc_filled = false;                // pc holds every plaintext of the model's layout
    Pool gpool;                            // private pool of the captured graphs
    std::map<std::string, ModelGraph> graphs;
    ~he_model() {
        for (auto &kv : graphs) {
            if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
            if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
        }
        graphs.clear();
        pc.pts.clear();
        gpool.release_all();
    }
};

struct he_ct {
    std::shared_ptr<Ctx> keep;   // declared first: destroyed after the buffers of x
    Ctx *c = nullptr;
    Cts x;
};

// check that x fits the model (layout, level); HE_EINVAL / HE_ELEVEL otherwise
void model_check_input(const he_model *m, const Cts &x);
// the model on x (CUDA graph per input shape when use_graph); output in a fresh buffer
Cts model_infer(he_model *m, const Cts &x, bool use_graph);
// a new C handle that shares x's buffer
he_ct *ct_wrap(Ctx *c, const Cts &x);
