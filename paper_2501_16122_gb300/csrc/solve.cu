// Preconditioned conjugate gradient for A x = b (paper Eq. 6) with the
// block-diagonal preconditioner of Eq. 7, in two precisions:
//
//  FP64:   every matvec in FP64.
//  MIXED:  iterative refinement.  Outer loop: r = b - A x with the FP64
//          operator (for white noise A is exactly the block-diagonal matrix
//          B of Eq. 7, so r = b - B x per pixel); inner loop: PCG on A e = r
//          with the FP32-product matvec to a relative tolerance of
//          max(1e-5, tol ||b|| / ||r||); x += e.
//
// CG scalars live on the device in FP64.  Every reduction uses a fixed grid
// and a fixed summation tree, so a solve is bitwise reproducible.  A device
// flag ends the iteration: kernels launched after convergence or a
// breakdown return at once.
#include <cmath>
#include <cstring>
#include <vector>

#include "bm_internal.cuh"

namespace bm {

namespace {

struct CgState {
    double rho;     // r . z
    double rr;      // r . r
    double bb;      // b . b
    double pq;      // p . A p
    double alpha, beta;
    double tol2;    // (tol ||b||)^2
    int done;       // 1 = converged, 2 = breakdown
    int iters;
};

constexpr int RB = kRedBlocks;
constexpr int RT = kRedThreads;

__device__ __forceinline__ double block_sum(double v, double* sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = RT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

// Sum of RB partials (fixed order) by one block.
__device__ __forceinline__ double sum_partials(const double* part, double* sh) {
    double v = 0.0;
    for (int i = threadIdx.x; i < RB; i += RT) v += part[i];
    return block_sum(v, sh);
}

template <int NC>
__device__ __forceinline__ void apply_M(const double* __restrict__ M, int64_t p, const double* r, double* z) {
    const double* m = M + p * NC * NC;
#pragma unroll
    for (int i = 0; i < NC; ++i) {
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < NC; ++j) s += m[i * NC + j] * r[j];
        z[i] = s;
    }
}

template <int NC>
__global__ void __launch_bounds__(RT) precond_kernel(const double* __restrict__ M, const double* __restrict__ r,
                                                     double* __restrict__ z, int64_t npix) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npix;
         p += (int64_t)gridDim.x * blockDim.x) {
        double rv[NC], zv[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) rv[c] = r[p * NC + c];
        apply_M<NC>(M, p, rv, zv);
#pragma unroll
        for (int c = 0; c < NC; ++c) z[p * NC + c] = zv[c];
    }
}

// Initial state from r (= b - A x0): z = M r, p = z; partials of r.z, r.r, b.b.
template <int NC>
__global__ void __launch_bounds__(RT) cg_init_kernel(const double* __restrict__ M, const double* __restrict__ b,
                                                     const double* __restrict__ r, double* __restrict__ z,
                                                     double* __restrict__ p, int64_t npix,
                                                     double* __restrict__ part) {
    __shared__ double sh[RT];
    double rz = 0.0, rr = 0.0, bb = 0.0;
    for (int64_t q = (int64_t)blockIdx.x * RT + threadIdx.x; q < npix; q += (int64_t)RB * RT) {
        double rv[NC], zv[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) rv[c] = r[q * NC + c];
        apply_M<NC>(M, q, rv, zv);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            z[q * NC + c] = zv[c];
            p[q * NC + c] = zv[c];
            rz += rv[c] * zv[c];
            rr += rv[c] * rv[c];
            const double bv = b[q * NC + c];
            bb += bv * bv;
        }
    }
    const double s0 = block_sum(rz, sh), s1 = block_sum(rr, sh), s2 = block_sum(bb, sh);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = s0;
        part[RB + blockIdx.x] = s1;
        part[2 * RB + blockIdx.x] = s2;
    }
}

__global__ void cg_init_finalize(const double* __restrict__ part, double tol, CgState* st) {
    __shared__ double sh[RT];
    const double rz = sum_partials(part, sh), rr = sum_partials(part + RB, sh),
                 bb = sum_partials(part + 2 * RB, sh);
    if (threadIdx.x == 0) {
        st->rho = rz;
        st->rr = rr;
        st->bb = bb;
        st->tol2 = tol * tol * bb;
        st->iters = 0;
        st->done = (rr <= st->tol2) ? 1 : 0;
    }
}

// Partials of p . q.
__global__ void __launch_bounds__(RT) dot_kernel(const double* __restrict__ a, const double* __restrict__ b,
                                                 int64_t n, const CgState* st, double* __restrict__ part) {
    __shared__ double sh[RT];
    if (st->done) return;
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * RT + threadIdx.x; i < n; i += (int64_t)RB * RT) s += a[i] * b[i];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void alpha_kernel(const double* __restrict__ part, CgState* st) {
    __shared__ double sh[RT];
    if (st->done) return;
    const double pq = sum_partials(part, sh);
    if (threadIdx.x == 0) {
        st->pq = pq;
        if (!(pq > 0.0) || !isfinite(pq) || !isfinite(st->rho)) {
            st->done = 2;
        } else {
            st->alpha = st->rho / pq;
        }
    }
}

// x += alpha p; r -= alpha q; z = M r; partials of r.r and r.z.
template <int NC>
__global__ void __launch_bounds__(RT) cg_update_kernel(const double* __restrict__ M, double* __restrict__ x,
                                                       double* __restrict__ r, double* __restrict__ z,
                                                       const double* __restrict__ p, const double* __restrict__ q,
                                                       int64_t npix, const CgState* st, double* __restrict__ part) {
    __shared__ double sh[RT];
    if (st->done) return;
    const double alpha = st->alpha;
    double rr = 0.0, rz = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * RT + threadIdx.x; i < npix; i += (int64_t)RB * RT) {
        double rv[NC], zv[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            x[i * NC + c] += alpha * p[i * NC + c];
            rv[c] = r[i * NC + c] - alpha * q[i * NC + c];
            r[i * NC + c] = rv[c];
        }
        apply_M<NC>(M, i, rv, zv);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            z[i * NC + c] = zv[c];
            rr += rv[c] * rv[c];
            rz += rv[c] * zv[c];
        }
    }
    const double s0 = block_sum(rr, sh), s1 = block_sum(rz, sh);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = s0;
        part[RB + blockIdx.x] = s1;
    }
}

__global__ void beta_kernel(const double* __restrict__ part, CgState* st) {
    __shared__ double sh[RT];
    if (st->done) return;
    const double rr = sum_partials(part, sh), rz = sum_partials(part + RB, sh);
    if (threadIdx.x == 0) {
        st->rr = rr;
        st->iters += 1;
        if (rr <= st->tol2) {
            st->done = 1;
        } else if (!isfinite(rz) || !isfinite(rr)) {
            st->done = 2;
        } else {
            st->beta = rz / st->rho;
            st->rho = rz;
        }
    }
}

__global__ void __launch_bounds__(RT) p_update_kernel(double* __restrict__ p, const double* __restrict__ z,
                                                      int64_t n, const CgState* st) {
    if (st->done) return;
    const double beta = st->beta;
    for (int64_t i = (int64_t)blockIdx.x * RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT)
        p[i] = z[i] + beta * p[i];
}

// r = b - B x per pixel (the FP64 white-noise operator), partial r.r.
template <int NC>
__global__ void __launch_bounds__(RT) block_residual_kernel(const double* __restrict__ B, const uint8_t* __restrict__ mask,
                                                            const double* __restrict__ b, const double* __restrict__ x,
                                                            double* __restrict__ r, int64_t npix,
                                                            double* __restrict__ part) {
    __shared__ double sh[RT];
    double rr = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * RT + threadIdx.x; i < npix; i += (int64_t)RB * RT) {
        const double* Bp = B + i * NC * NC;
        const bool keep = mask[i] == 0;
#pragma unroll
        for (int a = 0; a < NC; ++a) {
            double s = 0.0;
#pragma unroll
            for (int c = 0; c < NC; ++c) s += Bp[a * NC + c] * x[i * NC + c];
            const double v = keep ? b[i * NC + a] - s : 0.0;
            r[i * NC + a] = v;
            rr += v * v;
        }
    }
    rr = block_sum(rr, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = rr;
}

// r = b - q, partial r.r (q = A x from a matvec).
__global__ void __launch_bounds__(RT) sub_residual_kernel(const double* __restrict__ b, const double* __restrict__ q,
                                                          double* __restrict__ r, int64_t n, double* __restrict__ part) {
    __shared__ double sh[RT];
    double rr = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * RT + threadIdx.x; i < n; i += (int64_t)RB * RT) {
        const double v = b[i] - q[i];
        r[i] = v;
        rr += v * v;
    }
    rr = block_sum(rr, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = rr;
}

__global__ void sum_kernel(const double* __restrict__ part, double* __restrict__ out) {
    __shared__ double sh[RT];
    const double s = sum_partials(part, sh);
    if (threadIdx.x == 0) *out = s;
}

__global__ void axpy_kernel(double* __restrict__ x, const double* __restrict__ e, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] += e[i];
}

template <int NC>
__global__ void write_map_kernel(const double* __restrict__ x, const uint8_t* __restrict__ mask, int64_t npix,
                                 double* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npix; i += (int64_t)gridDim.x * blockDim.x)
#pragma unroll
        for (int c = 0; c < NC; ++c) out[i * NC + c] = mask[i] ? NAN : x[i * NC + c];
}

}  // namespace

void precond_apply(bm_precond* pc, const double* r, double* z, int64_t nrhs) {
    bm_context* ctx = pc->ctx;
    const int64_t npix = pc->p->npix;
    const int nc = pc->ncomp;
    const int grid = grid_for(ctx, (npix + RT - 1) / RT, 16);
    for (int64_t k = 0; k < nrhs; ++k) {
        const double* rk = r + k * npix * nc;
        double* zk = z + k * npix * nc;
        if (nc == 3) precond_kernel<3><<<grid, RT, 0, ctx->stream>>>(pc->Minv.get(), rk, zk, npix);
        else if (nc == 2) precond_kernel<2><<<grid, RT, 0, ctx->stream>>>(pc->Minv.get(), rk, zk, npix);
        else precond_kernel<1><<<grid, RT, 0, ctx->stream>>>(pc->Minv.get(), rk, zk, npix);
        BM_LAUNCH_CHECK();
    }
}

namespace {

// Device vectors and scalars of one PCG solve.
struct Cg {
    bm_precond* pc;
    int64_t npix, nvec;
    int nc;
    double *x, *r, *z, *p, *q, *part;
    CgState* st;
};

template <int NC>
void cg_start(Cg& cg, const double* b, const double* r0, double tol, cudaStream_t s) {
    cg_init_kernel<NC><<<RB, RT, 0, s>>>(cg.pc->Minv.get(), b, r0, cg.z, cg.p, cg.npix, cg.part);
    BM_LAUNCH_CHECK();
    cg_init_finalize<<<1, RT, 0, s>>>(cg.part, tol, cg.st);
    BM_LAUNCH_CHECK();
}

template <int NC>
void cg_iteration(Cg& cg, bm_pointing* p, bm_inv_noise* n, bm_precision prec, cudaStream_t s) {
    matvec(p, n, cg.pc, cg.p, cg.q, prec, 1);
    dot_kernel<<<RB, RT, 0, s>>>(cg.p, cg.q, cg.nvec, cg.st, cg.part);
    BM_LAUNCH_CHECK();
    alpha_kernel<<<1, RT, 0, s>>>(cg.part, cg.st);
    BM_LAUNCH_CHECK();
    cg_update_kernel<NC><<<RB, RT, 0, s>>>(cg.pc->Minv.get(), cg.x, cg.r, cg.z, cg.p, cg.q, cg.npix, cg.st, cg.part);
    BM_LAUNCH_CHECK();
    beta_kernel<<<1, RT, 0, s>>>(cg.part, cg.st);
    BM_LAUNCH_CHECK();
    p_update_kernel<<<grid_for(cg.pc->ctx, (cg.nvec + RT - 1) / RT, 16), RT, 0, s>>>(cg.p, cg.z, cg.nvec, cg.st);
    BM_LAUNCH_CHECK();
}

CgState read_state(bm_context* ctx, const CgState* st) {
    CgState h;
    BM_CUDA(cudaMemcpyAsync(ctx->h_pinned, st, sizeof(CgState), cudaMemcpyDeviceToHost, ctx->stream));
    BM_CUDA(cudaStreamSynchronize(ctx->stream));
    memcpy(&h, ctx->h_pinned, sizeof(CgState));
    return h;
}

// Loop control of the WHILE node below: loop[0] counts the iterations of the
// current graph launch (inc = 1 after an iteration, 0 before the first),
// loop[1] is their limit; the node goes on while the solve is not done and
// the limit is not reached.
__global__ void cg_loop_kernel(const CgState* __restrict__ st, int* __restrict__ loop, int inc,
                               cudaGraphConditionalHandle h) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int it = loop[0] + inc;
    loop[0] = it;
    cudaGraphSetConditional(h, (st->done == 0 && it < loop[1]) ? 1u : 0u);
}

// The PCG iterations of a solve as one CUDA graph: cg_loop_kernel decides
// whether to enter, then a WHILE node runs one iteration (matvec and CG
// updates) followed by cg_loop_kernel, until the state is done or the limit
// is reached; the host reads the state once afterwards instead of after
// every iteration.  Built on the context's side stream after one eager
// iteration (which makes every lazily built table and scratch buffer), for
// a solve on one process without kernel timing; rebuilt if a workspace has
// moved since (the graph holds their addresses).
struct CgLoop {
    cudaGraphExec_t exec = nullptr;
    uint64_t generation = 0;
    int64_t body_kernels = 0;
    bool ok = true;
    int* loop = nullptr;
    ~CgLoop() {
        if (exec) cudaGraphExecDestroy(exec);
    }
};

template <int NC>
void build_cg_loop(CgLoop& gl, Cg& cg, bm_pointing* p, bm_inv_noise* n, bm_precision prec) {
    bm_context* ctx = cg.pc->ctx;
    if (gl.exec) {
        cudaGraphExecDestroy(gl.exec);
        gl.exec = nullptr;
    }
    gl.loop = workspace_as<int>(ctx, "cg_loop", 2);
    gl.generation = ctx->ws_generation;
    cudaGraph_t graph = nullptr;
    BM_CUDA(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle h;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, graph, 0, cudaGraphCondAssignDefault);
    if (e == cudaSuccess)
        e = cudaStreamBeginCaptureToGraph(ctx->side, graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cg_loop_kernel<<<1, 32, 0, ctx->side>>>(cg.st, gl.loop, 0, h);
        e = cudaGetLastError();
        const cudaError_t e2 = cudaStreamEndCapture(ctx->side, &graph);
        if (e == cudaSuccess) e = e2;
    }
    cudaGraphNode_t first = nullptr;
    size_t nn = 1;
    if (e == cudaSuccess) e = cudaGraphGetNodes(graph, &first, &nn);
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t wnode = nullptr;
    if (e == cudaSuccess) e = cudaGraphAddNode(&wnode, graph, &first, nullptr, 1, &cp);
    if (e == cudaSuccess) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(ctx->side, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const int64_t before = bm_kernel_launches();
            cudaStream_t saved = ctx->stream;
            ctx->stream = ctx->side;  // the matvec launches on the context stream
            try {
                cg_iteration<NC>(cg, p, n, prec, ctx->side);
            } catch (...) {
                ctx->stream = saved;
                cudaStreamEndCapture(ctx->side, &body);
                cudaGraphDestroy(graph);
                throw;
            }
            ctx->stream = saved;
            gl.body_kernels = bm_kernel_launches() - before + 1;  // + the loop kernel
            count_launches(-(gl.body_kernels - 1));  // counted from the iterations that ran
            cg_loop_kernel<<<1, 32, 0, ctx->side>>>(cg.st, gl.loop, 1, h);
            e = cudaGetLastError();
            const cudaError_t e2 = cudaStreamEndCapture(ctx->side, &body);
            if (e == cudaSuccess) e = e2;
        }
    }
    // a workspace made while capturing would be a graph allocation: not usable
    if (e == cudaSuccess && ctx->ws_generation != gl.generation) e = cudaErrorStreamCaptureUnsupported;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&gl.exec, graph, 0);
    cudaGraphDestroy(graph);
    BM_CUDA(e);
}

// PCG on A x = b from x = 0 (x, r written into cg).  Returns iterations and the final state.
template <int NC>
CgState run_pcg(Cg& cg, bm_pointing* p, bm_inv_noise* n, const double* b, double tol, int maxiter,
                bm_precision prec, CgLoop* gl = nullptr) {
    bm_context* ctx = cg.pc->ctx;
    cudaStream_t s = ctx->stream;
    BM_CUDA(cudaMemsetAsync(cg.x, 0, sizeof(double) * cg.nvec, s));
    BM_CUDA(cudaMemcpyAsync(cg.r, b, sizeof(double) * cg.nvec, cudaMemcpyDeviceToDevice, s));
    cg_start<NC>(cg, b, cg.r, tol, s);
    CgState h = read_state(ctx, cg.st);
    int it = 0;
    if (!h.done && it < maxiter) {  // one iteration eagerly
        cg_iteration<NC>(cg, p, n, prec, s);
        ++it;
        h = read_state(ctx, cg.st);
    }
    const bool graph = gl && gl->ok && ctx->graphs && ctx->side && !ctx->allreduce && !ctx->timing;
    if (graph && !h.done && it < maxiter) {
        if (!gl->exec || gl->generation != ctx->ws_generation) {
            try {
                build_cg_loop<NC>(*gl, cg, p, n, prec);
            } catch (const Error&) {  // no conditional graph here: the host-driven loop below
                gl->ok = false;
                if (gl->exec) cudaGraphExecDestroy(gl->exec);
                gl->exec = nullptr;
                cudaGetLastError();
                clear_error();
            }
        }
        if (gl->exec) {
            const int hl[2] = {0, maxiter - it};
            BM_CUDA(cudaMemcpyAsync(gl->loop, hl, sizeof(hl), cudaMemcpyHostToDevice, s));
            BM_CUDA(cudaEventRecord(ctx->side_ev, s));
            BM_CUDA(cudaStreamWaitEvent(ctx->side, ctx->side_ev, 0));
            BM_CUDA(cudaGraphLaunch(gl->exec, ctx->side));
            BM_CUDA(cudaEventRecord(ctx->side_ev, ctx->side));
            BM_CUDA(cudaStreamWaitEvent(s, ctx->side_ev, 0));
            BM_CUDA(cudaMemcpyAsync(ctx->h_pinned + 16, gl->loop, sizeof(int), cudaMemcpyDeviceToHost, s));
            h = read_state(ctx, cg.st);  // synchronises the stream
            int ran = 0;
            memcpy(&ran, ctx->h_pinned + 16, sizeof(int));
            count_launches(1 + (int64_t)ran * gl->body_kernels);
            return h;
        }
    }
    for (; it < maxiter && !h.done; ++it) {
        cg_iteration<NC>(cg, p, n, prec, s);
        h = read_state(ctx, cg.st);
    }
    return h;
}

// ||b - A x|| into r with the exact operator (op = BM_PREC_FP64, or the
// double-float refinement operator kPrecRefine); returns ||r||^2.  For white
// noise A is block diagonal, so A x = B x per pixel in FP64 either way.
template <int NC>
double exact_residual(Cg& cg, bm_pointing* p, bm_inv_noise* n, const double* b, const double* x, double* r,
                      bm_precision op) {
    bm_context* ctx = cg.pc->ctx;
    cudaStream_t s = ctx->stream;
    if (diagonal_noise(n)) {
        block_residual_kernel<NC><<<RB, RT, 0, s>>>(cg.pc->B.get(), cg.pc->mask.get(), b, x, r, cg.npix, cg.part);
    } else {
        matvec(p, n, cg.pc, x, cg.q, op, 1);
        sub_residual_kernel<<<RB, RT, 0, s>>>(b, cg.q, r, cg.nvec, cg.part);
    }
    BM_LAUNCH_CHECK();
    double* out = reinterpret_cast<double*>(cg.st) + 16;  // scratch slot after the state
    sum_kernel<<<1, RT, 0, s>>>(cg.part, out);
    BM_LAUNCH_CHECK();
    BM_CUDA(cudaMemcpyAsync(ctx->h_pinned, out, sizeof(double), cudaMemcpyDeviceToHost, s));
    BM_CUDA(cudaStreamSynchronize(s));
    return ctx->h_pinned[0];
}

template <int NC>
bm_status solve_one(bm_pointing* p, bm_inv_noise* n, bm_precond* pc, const double* b, double* map_out,
                    double tol, int32_t maxiter, bm_precision prec, bm_solve_info* info) {
    bm_context* ctx = pc->ctx;
    cudaStream_t s = ctx->stream;
    Cg cg;
    cg.pc = pc;
    cg.npix = p->npix;
    cg.nc = NC;
    cg.nvec = p->npix * NC;
    cg.x = workspace_as<double>(ctx, "cg_x", cg.nvec);
    cg.r = workspace_as<double>(ctx, "cg_r", cg.nvec);
    cg.z = workspace_as<double>(ctx, "cg_z", cg.nvec);
    cg.p = workspace_as<double>(ctx, "cg_p", cg.nvec);
    cg.q = workspace_as<double>(ctx, "cg_q", cg.nvec);
    cg.part = workspace_as<double>(ctx, "cg_part", 3 * RB);
    cg.st = reinterpret_cast<CgState*>(workspace_as<double>(ctx, "cg_state", 32));
    double* xs = workspace_as<double>(ctx, "cg_xsol", cg.nvec);
    double* rs = workspace_as<double>(ctx, "cg_rsol", cg.nvec);

    bm_solve_info inf{};
    bm_status status = BM_OK;
    double bb = 0.0;
    CgLoop loop;
    {
        // ||b||^2 (as the residual of x = 0)
        BM_CUDA(cudaMemsetAsync(cg.x, 0, sizeof(double) * cg.nvec, s));
        sub_residual_kernel<<<RB, RT, 0, s>>>(b, cg.x, rs, cg.nvec, cg.part);
        BM_LAUNCH_CHECK();
        double* out = reinterpret_cast<double*>(cg.st) + 16;
        sum_kernel<<<1, RT, 0, s>>>(cg.part, out);
        BM_LAUNCH_CHECK();
        BM_CUDA(cudaMemcpyAsync(ctx->h_pinned, out, sizeof(double), cudaMemcpyDeviceToHost, s));
        BM_CUDA(cudaStreamSynchronize(s));
        bb = ctx->h_pinned[0];
    }
    const double bnorm = std::sqrt(bb);
    BM_CUDA(cudaMemsetAsync(xs, 0, sizeof(double) * cg.nvec, s));
    if (bb == 0.0) {
        inf.rel_residual = 0.0;
    } else if (prec == BM_PREC_FP64) {
        CgState h = run_pcg<NC>(cg, p, n, b, tol, maxiter, BM_PREC_FP64, &loop);
        BM_CUDA(cudaMemcpyAsync(xs, cg.x, sizeof(double) * cg.nvec, cudaMemcpyDeviceToDevice, s));
        inf.iterations = h.iters;
        if (h.done == 2) status = BM_ERR_BREAKDOWN;
    } else {
        // Mixed: outer exact residual (FP64 blocks for white noise, the
        // double-float operator for Toeplitz noise), inner FP32-product PCG
        // on the correction.
        // x starts at 0, so the first residual is b itself (zero on masked pixels).
        BM_CUDA(cudaMemcpyAsync(rs, b, sizeof(double) * cg.nvec, cudaMemcpyDeviceToDevice, s));
        double rr = bb;
        int inner_total = 0, outer = 0;
        const int max_outer = 30;
        while (std::sqrt(rr) > tol * bnorm && inner_total < maxiter && outer < max_outer) {
            const double inner_tol = std::max(1e-6, 0.5 * tol * bnorm / std::sqrt(rr));
            CgState h = run_pcg<NC>(cg, p, n, rs, std::min(inner_tol, 0.5), maxiter - inner_total, BM_PREC_MIXED,
                                    &loop);
            inner_total += h.iters;
            ++outer;
            if (h.done == 2 && h.iters == 0) { status = BM_ERR_BREAKDOWN; break; }
            axpy_kernel<<<grid_for(ctx, (cg.nvec + 255) / 256, 16), 256, 0, s>>>(xs, cg.x, cg.nvec);
            BM_LAUNCH_CHECK();
            const double rr_new = exact_residual<NC>(cg, p, n, b, xs, rs, kPrecRefine);
            if (!(rr_new < rr)) { rr = rr_new; break; }  // stagnation
            rr = rr_new;
        }
        inf.iterations = inner_total;
        inf.outer_iterations = outer;
        inf.rel_residual = std::sqrt(rr) / bnorm;  // the last outer residual is the final one
    }
    if (bb != 0.0 && prec == BM_PREC_FP64) {
        // Final residual recomputed with the FP64 operator (the recurrence drifts).
        inf.rel_residual = std::sqrt(exact_residual<NC>(cg, p, n, b, xs, rs, BM_PREC_FP64)) / bnorm;
    }
    if (status == BM_OK && !(inf.rel_residual <= tol)) status = BM_ERR_NOT_CONVERGED;
    inf.status = status;
    const int threads = 256;
    write_map_kernel<NC><<<grid_for(ctx, (cg.npix + threads - 1) / threads, 16), threads, 0, s>>>(
        xs, pc->mask.get(), cg.npix, map_out);
    BM_LAUNCH_CHECK();
    BM_CUDA(cudaStreamSynchronize(s));
    if (info) *info = inf;
    return status;
}

}  // namespace

bm_status pcg_solve(bm_pointing* p, bm_inv_noise* n, bm_precond* pc, const void* tod, bm_dtype dt,
                    int32_t nrhs, double* map_out, double tol, int32_t maxiter, bm_precision prec,
                    bm_solve_info* info) {
    bm_context* ctx = p->ctx;
    const int nc = p->ncomp;
    const int64_t nvec = p->npix * nc;
    if (nrhs > 1 && n->kind == 0 && prec == BM_PREC_MIXED && !ctx->allreduce) {
        const bm_status st = batched_white_solve(p, n, pc, tod, dt, nrhs, map_out, tol, maxiter, info);
        if (st != BM_OK) set_error("at least one right-hand side did not converge (%s)", bm_status_string(st));
        return st;
    }
    double* b = workspace_as<double>(ctx, "solve_b", nvec);
    bm_status first = BM_OK;
    for (int32_t r = 0; r < nrhs; ++r) {
        const void* tr = tod ? static_cast<const char*>(tod) + (size_t)r * p->nsamples * (dt == BM_F32 ? 4 : 8)
                             : nullptr;  // the TOD sorted along with the pointing
        rhs(p, n, pc, tr, dt, 1, b, prec == BM_PREC_MIXED);
        bm_solve_info* ir = info ? info + r : nullptr;
        bm_status st;
        if (nc == 3) st = solve_one<3>(p, n, pc, b, map_out + r * nvec, tol, maxiter, prec, ir);
        else if (nc == 2) st = solve_one<2>(p, n, pc, b, map_out + r * nvec, tol, maxiter, prec, ir);
        else st = solve_one<1>(p, n, pc, b, map_out + r * nvec, tol, maxiter, prec, ir);
        if (first == BM_OK && st != BM_OK) first = st;
    }
    if (first != BM_OK) set_error("at least one right-hand side did not converge (%s)", bm_status_string(first));
    return first;
}

}  // namespace bm
