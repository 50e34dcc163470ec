// batch.cu -- CUDA-graph replay of the batched shoot (uneven refinement
// batches, Sec. 4 / Sec. 3.3): the kernel sequence of one lens_shoot_batches
// call is captured once per (sizes, pointers, flags) key and replayed.
#include <vector>

#include "walk_shared.cuh"

namespace lens {

lens_status enqueue_shoot(lens_tree* t, const ShootPlan& plan, const void* dx, const void* dy, int dtype,
                          void* const out[5], int flags, cudaStream_t s);

struct GraphEntry {
    int64_t n, nb;
    uint64_t ng;
    const void *dx, *dy;
    int dtype, flags;
    int group_rays, walk;  // the tree's settings when captured
    void* out[5];
    void* scratch;
    int64_t kernels;  // kernel nodes in the graph, added to the launch counter per replay
    cudaGraphExec_t exec;
};

// Number of kernel nodes in a captured graph.
static int64_t count_kernel_nodes(cudaGraph_t graph)
{
    size_t n = 0;
    if (cudaGraphGetNodes(graph, nullptr, &n) != cudaSuccess || n == 0) return 0;
    std::vector<cudaGraphNode_t> nodes(n);
    if (cudaGraphGetNodes(graph, nodes.data(), &n) != cudaSuccess) return 0;
    int64_t k = 0;
    for (size_t i = 0; i < n; ++i) {
        cudaGraphNodeType ty;
        if (cudaGraphNodeGetType(nodes[i], &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++k;
    }
    return k;
}

void free_graphs(lens_tree* t)
{
    for (GraphEntry* g : t->graphs) {
        if (g->exec) cudaGraphExecDestroy(g->exec);
        delete g;
    }
    t->graphs.clear();
}

lens_status graph_shoot_batches(lens_tree* t, int64_t nb, const int64_t* off, const double* orig,
                                const void* dx, const void* dy, int dtype, void* const out[5],
                                int flags, cudaStream_t s)
{
    ShootPlan plan;
    LENS_TRY(upload_batches(t, nb, off, orig, s, &plan, shoot_max_r(t, flags)));
    t->grp_n = -1;  // a replay regroups in the scratch without telling the host
    for (GraphEntry* g : t->graphs) {
        bool same = g->n == plan.n && g->nb == plan.nb && g->ng == plan.ng && g->dx == dx && g->dy == dy &&
                    g->dtype == dtype && g->flags == flags && g->scratch == t->ray_scratch.ptr &&
                    g->group_rays == t->group_rays && g->walk == t->walk_mode;
        for (int q = 0; q < 5 && same; ++q) same = g->out[q] == out[q];
        if (same) {
            LENS_TRY(wait_built(t, s));  // the graph itself holds no wait
            LENS_CUDA(cudaGraphLaunch(g->exec, s));
            note_launches(g->kernels);
            return LENS_OK;
        }
    }
    // first use of this key: run eagerly, then capture for the next calls
    LENS_TRY(enqueue_shoot(t, plan, dx, dy, dtype, out, flags, s));
    cudaStream_t cs;
    LENS_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaStreamDestroy(cs);
        return lens_cuda_check(e, "cudaStreamBeginCapture");
    }
    const int64_t before = lens_kernel_launches();
    lens_status st = enqueue_shoot(t, plan, dx, dy, dtype, out, flags, cs);
    note_launches(before - lens_kernel_launches());  // capture records kernels without running them
    e = cudaStreamEndCapture(cs, &graph);
    cudaStreamDestroy(cs);
    if (st != LENS_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return lens_cuda_check(e, "cudaStreamEndCapture");
    const int64_t kernels = count_kernel_nodes(graph);
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return lens_cuda_check(e, "cudaGraphInstantiate");
    GraphEntry* g = new GraphEntry{plan.n, plan.nb, plan.ng, dx, dy, dtype, flags, t->group_rays, t->walk_mode, {},
                                  t->ray_scratch.ptr, kernels, exec};
    for (int q = 0; q < 5; ++q) g->out[q] = out[q];
    t->graphs.push_back(g);
    return LENS_OK;
}

}  // namespace lens
