// extern "C" entry points of liblider.so (declared in include/lider.h) and the
// thread-local error message.  No C++ exception crosses this boundary.
#include <algorithm>
#include <exception>
#include <string>
#include <vector>

#include "lider_internal.cuh"

namespace lider {

namespace {
thread_local std::string g_last_error;
}

const char* g_last_error_ptr() { return g_last_error.c_str(); }

void set_error(const std::string& msg) { g_last_error = msg; }

int fail(int code, const std::string& msg) {
    set_error(msg);
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    cudaGetLastError();   // clear a non-sticky error so the next call starts clean
    set_error(std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
    return e == cudaErrorMemoryAllocation ? LIDER_ENOMEM : LIDER_ECUDA;
}

int build_entry(const float*, int64_t, int32_t, const float*, int32_t, const lider_cluster_params*, const float*,
                const float*, const lider_params*, void*, lider_index**);
void destroy_index(lider_index*);
int search_entry(const lider_index*, const float*, int64_t, int, int, int64_t*, float*, const lider_trace*,
                 lider_search_stats*, void*);
int search_scratch_entry(const lider_index*, int64_t, int, int, size_t*);
bool tuning_valid(const lider_tuning&);
int autotune_entry(lider_index*, const float*, int64_t, int, int, int, lider_tuning*, double*, void*);
int server_create_entry(const lider_index*, const lider_server_params*, lider_server**);
int server_submit_entry(lider_server*, const float*, int64_t, int32_t, int64_t*, float*, int64_t*);
int server_wait_entry(lider_server*, int64_t, double);
int server_stats_entry(lider_server*, lider_server_counters*);
int server_latencies_entry(lider_server*, double*, int64_t, int32_t, int64_t*);
void server_destroy_entry(lider_server*);
int search_host_entry(const lider_index*, const float*, int64_t, int, int, int64_t*, float*,
                      lider_search_stats*, void*);

template <class F>
int guarded(F&& f) {
    try {
        return f();
    } catch (const std::bad_alloc&) {
        return fail(LIDER_ENOMEM, "host allocation failed");
    } catch (const std::exception& e) {
        return fail(LIDER_ECUDA, std::string("internal error: ") + e.what());
    } catch (...) {
        return fail(LIDER_ECUDA, "internal error");
    }
}

}  // namespace lider

using namespace lider;

extern "C" {

int lider_build(const float* corpus, int64_t n, int32_t d, const lider_cluster_params* cluster, const float* A,
                const float* b, const lider_params* params, void* stream, lider_index** out) {
    return guarded([&]() -> int {
        if (!cluster) {
            if (out) *out = nullptr;
            return fail(LIDER_EINVAL, "lider_build: cluster is NULL");
        }
        return build_entry(corpus, n, d, nullptr, 0, cluster, A, b, params, stream, out);
    });
}

int lider_build_centroids(const float* corpus, int64_t n, int32_t d, const float* centroids, int32_t n_clusters,
                          const float* A, const float* b, const lider_params* params, void* stream,
                          lider_index** out) {
    return guarded([&] {
        return build_entry(corpus, n, d, centroids, n_clusters, nullptr, A, b, params, stream, out);
    });
}

int lider_get_build_info(const lider_index* index, lider_build_info* info) {
    if (!index || !info) return fail(LIDER_EINVAL, "lider_get_build_info: NULL argument");
    *info = lider_build_info{};
    info->clustered = index->clustered ? 1 : 0;
    info->projections_drawn = index->projections_drawn ? 1 : 0;
    info->cluster = index->cluster;
    if (index->clustered)
        info->train_rows = index->cluster.kmeans_sample == 0 ? index->g.n
                                                              : std::min<int64_t>(index->cluster.kmeans_sample, index->g.n);
    int32_t empty = 0;
    for (int j = 0; j < index->g.ncl; ++j) empty += index->h_cl_off[j + 1] == index->h_cl_off[j];
    info->empty_clusters = empty;
    info->kmeans_ms = index->kmeans_ms;
    info->build_ms = index->build_ms;
    return LIDER_OK;
}

int lider_export_centroids(const lider_index* index, float* centroids_host) {
    return guarded([&]() -> int {
        if (!index || !centroids_host) return fail(LIDER_EINVAL, "lider_export_centroids: NULL argument");
        LIDER_CUDA_TRY(cudaMemcpy(centroids_host, index->g.C, (size_t)index->g.ncl * index->g.d * sizeof(float),
                                  cudaMemcpyDeviceToHost));
        return LIDER_OK;
    });
}

int lider_export_assignment(const lider_index* index, int32_t* asg_host) {
    return guarded([&]() -> int {
        if (!index || !asg_host) return fail(LIDER_EINVAL, "lider_export_assignment: NULL argument");
        const Geometry& g = index->g;
        std::vector<int64_t> orig((size_t)g.n);
        LIDER_CUDA_TRY(cudaMemcpy(orig.data(), g.orig_id, (size_t)g.n * sizeof(int64_t), cudaMemcpyDeviceToHost));
        for (int j = 0; j < g.ncl; ++j)
            for (int64_t r = index->h_cl_off[j]; r < index->h_cl_off[j + 1]; ++r) {
                if (orig[r] < 0 || orig[r] >= g.n) return fail(LIDER_ECUDA, "lider_export_assignment: corrupt id");
                asg_host[orig[r]] = j;
            }
        return LIDER_OK;
    });
}

int lider_export_projections(const lider_index* index, float* A_host, float* b_host) {
    return guarded([&]() -> int {
        if (!index) return fail(LIDER_EINVAL, "lider_export_projections: index is NULL");
        const Geometry& g = index->g;
        if (A_host)
            LIDER_CUDA_TRY(cudaMemcpy(A_host, g.A, (size_t)g.H * g.d * sizeof(float), cudaMemcpyDeviceToHost));
        if (b_host) LIDER_CUDA_TRY(cudaMemcpy(b_host, g.bproj, (size_t)g.H * sizeof(float), cudaMemcpyDeviceToHost));
        return LIDER_OK;
    });
}

int lider_search(const lider_index* index, const float* queries, int64_t nq, int32_t k, int32_t c,
                 int64_t* out_ids, float* out_scores, lider_search_stats* stats, void* stream) {
    return guarded([&] {
        return search_entry(index, queries, nq, k, c, out_ids, out_scores, nullptr, stats, stream);
    });
}

int lider_search_trace(const lider_index* index, const float* queries, int64_t nq, int32_t k, int32_t c,
                       int64_t* out_ids, float* out_scores, const lider_trace* trace, lider_search_stats* stats,
                       void* stream) {
    return guarded([&] {
        return search_entry(index, queries, nq, k, c, out_ids, out_scores, trace, stats, stream);
    });
}

int lider_search_host(const lider_index* index, const float* queries_host, int64_t nq, int32_t k, int32_t c,
                      int64_t* ids_host, float* scores_host, lider_search_stats* stats, void* stream) {
    return guarded([&] {
        return search_host_entry(index, queries_host, nq, k, c, ids_host, scores_host, stats, stream);
    });
}

int lider_search_scratch_bytes(const lider_index* index, int64_t nq, int32_t k, int32_t c, size_t* bytes) {
    return guarded([&] { return search_scratch_entry(index, nq, k, c, bytes); });
}

int lider_server_create(const lider_index* index, const lider_server_params* params, lider_server** out) {
    return guarded([&] { return server_create_entry(index, params, out); });
}

int lider_server_submit(lider_server* server, const float* queries_host, int64_t nq, int32_t k,
                        int64_t* ids_host, float* scores_host, int64_t* ticket) {
    return guarded([&] { return server_submit_entry(server, queries_host, nq, k, ids_host, scores_host, ticket); });
}

int lider_server_wait(lider_server* server, int64_t ticket, double timeout_s) {
    return guarded([&] { return server_wait_entry(server, ticket, timeout_s); });
}

int lider_server_stats(lider_server* server, lider_server_counters* stats) {
    return guarded([&] { return server_stats_entry(server, stats); });
}

int lider_server_latencies(lider_server* server, double* out_ms, int64_t cap, int32_t clear, int64_t* total) {
    return guarded([&] { return server_latencies_entry(server, out_ms, cap, clear, total); });
}

void lider_server_destroy(lider_server* server) {
    try {
        server_destroy_entry(server);
    } catch (...) {
    }
}

int lider_get_tuning(const lider_index* index, lider_tuning* tuning) {
    if (!index || !tuning) return fail(LIDER_EINVAL, "lider_get_tuning: NULL argument");
    *tuning = index->tune;
    return LIDER_OK;
}

int lider_set_tuning(lider_index* index, const lider_tuning* tuning) {
    if (!index || !tuning) return fail(LIDER_EINVAL, "lider_set_tuning: NULL argument");
    if (!tuning_valid(*tuning)) return fail(LIDER_EINVAL, "lider_set_tuning: a value is outside its allowed set");
    index->tune = *tuning;
    return LIDER_OK;
}

int lider_autotune(lider_index* index, const float* queries, int64_t nq, int32_t k, int32_t c, int32_t reps,
                   lider_tuning* chosen, double* best_ms, void* stream) {
    return guarded([&] { return autotune_entry(index, queries, nq, k, c, reps, chosen, best_ms, stream); });
}

int lider_index_info(const lider_index* index, int64_t* n, int32_t* d, int32_t* n_clusters, lider_params* params) {
    if (!index) return fail(LIDER_EINVAL, "lider_index_info: index is NULL");
    if (n) *n = index->g.n;
    if (d) *d = index->g.d;
    if (n_clusters) *n_clusters = index->g.ncl;
    if (params) *params = index->params;
    return LIDER_OK;
}

int lider_cluster_offsets(const lider_index* index, int64_t* offsets_host) {
    if (!index || !offsets_host) return fail(LIDER_EINVAL, "lider_cluster_offsets: NULL argument");
    for (size_t i = 0; i < index->h_cl_off.size(); ++i) offsets_host[i] = index->h_cl_off[i];
    return LIDER_OK;
}

int lider_export_array(const lider_index* index, int32_t cluster, int32_t array, uint64_t* keys_host,
                       int64_t* ids_host) {
    return guarded([&]() -> int {
        if (!index || !keys_host || !ids_host) return fail(LIDER_EINVAL, "lider_export_array: NULL argument");
        const Geometry& g = index->g;
        if (cluster < 0 || cluster >= g.ncl || array < 0 || array >= g.L)
            return fail(LIDER_EINVAL, "lider_export_array: cluster or array out of range");
        const int64_t base = index->h_cl_off[cluster], n_c = index->h_cl_off[cluster + 1] - base;
        if (n_c == 0) return LIDER_OK;
        LIDER_CUDA_TRY(cudaMemcpy(keys_host, g.keys + (int64_t)array * g.n + base, n_c * 8, cudaMemcpyDeviceToHost));
        std::vector<int32_t> pos(n_c);
        std::vector<int64_t> orig(n_c);
        LIDER_CUDA_TRY(cudaMemcpy(pos.data(), g.pos + (int64_t)array * g.n + base, n_c * 4, cudaMemcpyDeviceToHost));
        LIDER_CUDA_TRY(cudaMemcpy(orig.data(), g.orig_id + base, n_c * 8, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < n_c; ++i) {
            if (pos[i] < 0 || pos[i] >= n_c) return fail(LIDER_ECUDA, "lider_export_array: corrupt position");
            ids_host[i] = orig[pos[i]];
        }
        return LIDER_OK;
    });
}

int lider_export_rmi(const lider_index* index, int32_t cluster, int32_t array, uint64_t* minmax_host,
                     double* root_host, double* leaf_host, int32_t* err_host) {
    return guarded([&]() -> int {
        if (!index) return fail(LIDER_EINVAL, "lider_export_rmi: index is NULL");
        const Geometry& g = index->g;
        if (cluster < 0 || cluster >= g.ncl || array < 0 || array >= g.L)
            return fail(LIDER_EINVAL, "lider_export_rmi: cluster or array out of range");
        RmiRoot rt;
        LIDER_CUDA_TRY(cudaMemcpy(&rt, g.root + (int64_t)cluster * g.L + array, sizeof(rt), cudaMemcpyDeviceToHost));
        if (minmax_host) { minmax_host[0] = rt.x_min; minmax_host[1] = rt.x_max; }
        if (root_host) { root_host[0] = rt.a0; root_host[1] = rt.b0; }
        if (leaf_host || err_host) {
            std::vector<RmiLeaf> lv(g.F);
            LIDER_CUDA_TRY(cudaMemcpy(lv.data(), g.leaf + ((int64_t)cluster * g.L + array) * g.F,
                                      sizeof(RmiLeaf) * g.F, cudaMemcpyDeviceToHost));
            for (int f = 0; f < g.F; ++f) {
                if (leaf_host) { leaf_host[2 * f] = lv[f].a; leaf_host[2 * f + 1] = lv[f].b; }
                if (err_host) { err_host[2 * f] = lv[f].lo; err_host[2 * f + 1] = lv[f].hi; }
            }
        }
        return LIDER_OK;
    });
}

void lider_free(lider_index* index) {
    try {
        destroy_index(index);
    } catch (...) {
    }
}

const char* lider_last_error(void) { return g_last_error_ptr(); }

}  // extern "C"
