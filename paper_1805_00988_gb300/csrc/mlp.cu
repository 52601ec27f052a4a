// mlp.cu -- the plan cost model: a small MLP (d_in -> h -> h -> 1, ReLU)
// predicting the log of a segment's run time under a plan variant, with
// hand-written forward, backward (mean-squared error) and Adam kernels.
//
// Parameters are one flat FP32 vector: W1 (d_in x h, row-major), b1 (h),
// W2 (h x h), b2 (h), W3 (h x 1), b3 (1).  Every reduction over rows runs in
// a fixed order (one thread per weight looping over the rows), so gradients
// are bit-reproducible.
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.cuh"

struct qsim_mlp;

namespace qsim {

namespace {

struct Off {
    int64_t w1, b1, w2, b2, w3, b3, total;
};

Off offsets(int d, int h)
{
    Off o;
    o.w1 = 0;
    o.b1 = o.w1 + (int64_t)d * h;
    o.w2 = o.b1 + h;
    o.b2 = o.w2 + (int64_t)h * h;
    o.w3 = o.b2 + h;
    o.b3 = o.w3 + h;
    o.total = o.b3 + 1;
    return o;
}

// z = in (rows x din) @ W (din x dout) + b ; a = relu(z) (if relu)
__global__ void k_dense(const float *__restrict__ in, int64_t rows, int din, const float *__restrict__ W,
                        const float *__restrict__ b, int dout, float *__restrict__ z, float *__restrict__ a)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= rows * dout) return;
    const int64_t r = e / dout;
    const int j = (int)(e % dout);
    float s = b[j];
    for (int i = 0; i < din; ++i) s = fmaf(in[r * din + i], W[(int64_t)i * dout + j], s);
    z[e] = s;
    if (a) a[e] = s > 0.f ? s : 0.f;
}

// dy = 2 / R (y - t)
__global__ void k_dloss(const float *__restrict__ y, const float *__restrict__ t, int64_t rows, float *__restrict__ dy)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < rows) dy[r] = (2.0f / (float)rows) * (y[r] - t[r]);
}

// gW[i][j] = sum_r in[r][i] * d[r][j],  gb[j] = sum_r d[r][j]   (one thread per weight)
__global__ void k_wgrad(const float *__restrict__ in, const float *__restrict__ d, int64_t rows, int din, int dout,
                        float *__restrict__ gW, float *__restrict__ gb)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < din * dout) {
        const int i = e / dout, j = e % dout;
        float s = 0.f;
        for (int64_t r = 0; r < rows; ++r) s = fmaf(in[r * din + i], d[r * dout + j], s);
        gW[e] = s;
    } else if (e < din * dout + dout) {
        const int j = e - din * dout;
        float s = 0.f;
        for (int64_t r = 0; r < rows; ++r) s += d[r * dout + j];
        gb[j] = s;
    }
}

// din_grad[r][i] = (sum_j d[r][j] W[i][j]) * (zprev[r][i] > 0)
__global__ void k_backprop(const float *__restrict__ d, const float *__restrict__ W, const float *__restrict__ zprev,
                           int64_t rows, int din, int dout, float *__restrict__ out)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= rows * din) return;
    const int64_t r = e / din;
    const int i = (int)(e % din);
    float s = 0.f;
    for (int j = 0; j < dout; ++j) s = fmaf(d[r * dout + j], W[(int64_t)i * dout + j], s);
    out[e] = zprev[e] > 0.f ? s : 0.f;
}

// Adam (Kingma & Ba 2015), bias-corrected
__global__ void k_adam(float *__restrict__ th, const float *__restrict__ g, float *__restrict__ m, float *__restrict__ v,
                       int64_t n, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float mi = b1 * m[i] + (1.f - b1) * g[i];
    const float vi = b2 * v[i] + (1.f - b2) * g[i] * g[i];
    m[i] = mi;
    v[i] = vi;
    th[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// mean of (y - t)^2 in one CTA, fixed order
__global__ void k_mse(const float *__restrict__ y, const float *__restrict__ t, int64_t rows, float *__restrict__ out)
{
    __shared__ double sh[256];
    double s = 0.0;
    for (int64_t r = threadIdx.x; r < rows; r += 256) {
        const double e = (double)y[r] - (double)t[r];
        s += e * e;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = (float)(sh[0] / (double)rows);
}

unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

}  // namespace qsim

using namespace qsim;

struct qsim_mlp {
    int d = 0, h = 0;
    Off off{};
    cudaStream_t stream = nullptr;
    bool owns_stream = false;
    float *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    int t = 0;
    // activations for up to cap rows
    int64_t cap = 0;
    float *x = nullptr, *tgt = nullptr, *z1 = nullptr, *a1 = nullptr, *z2 = nullptr, *a2 = nullptr, *y = nullptr;
    float *d2 = nullptr, *d1 = nullptr, *dy = nullptr, *loss = nullptr;
};

static void mlp_free_acts(qsim_mlp *m)
{
    float **ptrs[] = {&m->x, &m->tgt, &m->z1, &m->a1, &m->z2, &m->a2, &m->y, &m->d2, &m->d1, &m->dy};
    for (float **p : ptrs) {
        if (*p) cudaFree(*p);
        *p = nullptr;
    }
    m->cap = 0;
}

static int mlp_reserve(qsim_mlp *m, int64_t rows)
{
    if (rows <= m->cap) return SIM_OK;
    mlp_free_acts(m);
    const int64_t R = rows;
    QSIM_CUDA(cudaMalloc((void **)&m->x, sizeof(float) * R * m->d));
    QSIM_CUDA(cudaMalloc((void **)&m->tgt, sizeof(float) * R));
    QSIM_CUDA(cudaMalloc((void **)&m->z1, sizeof(float) * R * m->h));
    QSIM_CUDA(cudaMalloc((void **)&m->a1, sizeof(float) * R * m->h));
    QSIM_CUDA(cudaMalloc((void **)&m->z2, sizeof(float) * R * m->h));
    QSIM_CUDA(cudaMalloc((void **)&m->a2, sizeof(float) * R * m->h));
    QSIM_CUDA(cudaMalloc((void **)&m->y, sizeof(float) * R));
    QSIM_CUDA(cudaMalloc((void **)&m->d2, sizeof(float) * R * m->h));
    QSIM_CUDA(cudaMalloc((void **)&m->d1, sizeof(float) * R * m->h));
    QSIM_CUDA(cudaMalloc((void **)&m->dy, sizeof(float) * R));
    m->cap = R;
    return SIM_OK;
}

// forward on m->x (rows already in place); leaves y in m->y
static int mlp_fwd(qsim_mlp *m, int64_t rows)
{
    const int T = 256;
    const Off &o = m->off;
    k_dense<<<blocks_for(rows * m->h, T), T, 0, m->stream>>>(m->x, rows, m->d, m->theta + o.w1, m->theta + o.b1, m->h,
                                                             m->z1, m->a1);
    k_dense<<<blocks_for(rows * m->h, T), T, 0, m->stream>>>(m->a1, rows, m->h, m->theta + o.w2, m->theta + o.b2, m->h,
                                                             m->z2, m->a2);
    k_dense<<<blocks_for(rows, T), T, 0, m->stream>>>(m->a2, rows, m->h, m->theta + o.w3, m->theta + o.b3, 1, m->y,
                                                      nullptr);
    QSIM_CUDA(cudaGetLastError());
    return SIM_OK;
}

// gradient of the MSE loss into m->grad; loss into m->loss
static int mlp_bwd(qsim_mlp *m, int64_t rows)
{
    const int T = 256;
    const Off &o = m->off;
    const int d = m->d, h = m->h;
    k_mse<<<1, 256, 0, m->stream>>>(m->y, m->tgt, rows, m->loss);
    k_dloss<<<blocks_for(rows, T), T, 0, m->stream>>>(m->y, m->tgt, rows, m->dy);
    k_wgrad<<<blocks_for(h + 1, T), T, 0, m->stream>>>(m->a2, m->dy, rows, h, 1, m->grad + o.w3, m->grad + o.b3);
    k_backprop<<<blocks_for(rows * h, T), T, 0, m->stream>>>(m->dy, m->theta + o.w3, m->z2, rows, h, 1, m->d2);
    k_wgrad<<<blocks_for(h * h + h, T), T, 0, m->stream>>>(m->a1, m->d2, rows, h, h, m->grad + o.w2, m->grad + o.b2);
    k_backprop<<<blocks_for(rows * h, T), T, 0, m->stream>>>(m->d2, m->theta + o.w2, m->z1, rows, h, h, m->d1);
    k_wgrad<<<blocks_for(d * h + h, T), T, 0, m->stream>>>(m->x, m->d1, rows, d, h, m->grad + o.w1, m->grad + o.b1);
    QSIM_CUDA(cudaGetLastError());
    return SIM_OK;
}

static int mlp_load_xy(qsim_mlp *m, const float *x, const float *t, int64_t rows, int on_device)
{
    if (int rc = mlp_reserve(m, rows)) return rc;
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    QSIM_CUDA(cudaMemcpyAsync(m->x, x, sizeof(float) * rows * m->d, k, m->stream));
    if (t) QSIM_CUDA(cudaMemcpyAsync(m->tgt, t, sizeof(float) * rows, k, m->stream));
    return SIM_OK;
}

extern "C" {

int sim_mlp_param_count(int d_in, int hidden) { return (int)offsets(d_in, hidden).total; }

int sim_mlp_create(int d_in, int hidden, void *stream, qsim_mlp **out)
{
    set_error("");
    if (!out || d_in < 1 || d_in > 256 || hidden < 1 || hidden > 256)
        return fail(SIM_EINVAL, "sim_mlp_create: d_in and hidden must be in 1..256");
    qsim_mlp *m = new qsim_mlp();
    m->d = d_in;
    m->h = hidden;
    m->off = offsets(d_in, hidden);
    int rc = SIM_OK;
    do {
        if (stream) {
            m->stream = (cudaStream_t)stream;
        } else {
            if (cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking) != cudaSuccess) {
                rc = cuda_fail(cudaGetLastError(), "mlp stream");
                break;
            }
            m->owns_stream = true;
        }
        const size_t b = sizeof(float) * m->off.total;
        if (cudaMalloc((void **)&m->theta, b) != cudaSuccess || cudaMalloc((void **)&m->grad, b) != cudaSuccess ||
            cudaMalloc((void **)&m->m, b) != cudaSuccess || cudaMalloc((void **)&m->v, b) != cudaSuccess ||
            cudaMalloc((void **)&m->loss, sizeof(float)) != cudaSuccess) {
            rc = cuda_fail(cudaGetLastError(), "mlp allocation");
            break;
        }
        cudaMemset(m->theta, 0, b);
        cudaMemset(m->m, 0, b);
        cudaMemset(m->v, 0, b);
    } while (0);
    if (rc) {
        sim_mlp_destroy(m);
        return rc;
    }
    *out = m;
    return SIM_OK;
}

int sim_mlp_destroy(qsim_mlp *m)
{
    if (!m) return SIM_OK;
    if (m->stream) cudaStreamSynchronize(m->stream);
    mlp_free_acts(m);
    float *p[] = {m->theta, m->grad, m->m, m->v, m->loss};
    for (float *q : p)
        if (q) cudaFree(q);
    if (m->owns_stream && m->stream) cudaStreamDestroy(m->stream);
    delete m;
    return SIM_OK;
}

int sim_mlp_set_params(qsim_mlp *m, const float *theta_host)
{
    if (!m || !theta_host) return fail(SIM_EINVAL, "sim_mlp_set_params: bad arguments");
    const size_t b = sizeof(float) * m->off.total;
    QSIM_CUDA(cudaMemcpyAsync(m->theta, theta_host, b, cudaMemcpyHostToDevice, m->stream));
    QSIM_CUDA(cudaMemsetAsync(m->m, 0, b, m->stream));
    QSIM_CUDA(cudaMemsetAsync(m->v, 0, b, m->stream));
    QSIM_CUDA(cudaStreamSynchronize(m->stream));
    m->t = 0;
    return SIM_OK;
}

int sim_mlp_get_params(qsim_mlp *m, float *theta_host)
{
    if (!m || !theta_host) return fail(SIM_EINVAL, "sim_mlp_get_params: bad arguments");
    QSIM_CUDA(cudaMemcpyAsync(theta_host, m->theta, sizeof(float) * m->off.total, cudaMemcpyDeviceToHost, m->stream));
    QSIM_CUDA(cudaStreamSynchronize(m->stream));
    return SIM_OK;
}

int sim_mlp_forward(qsim_mlp *m, const float *x, int64_t rows, float *y, int on_device)
{
    if (!m || !x || !y || rows < 1) return fail(SIM_EINVAL, "sim_mlp_forward: bad arguments");
    if (int rc = mlp_load_xy(m, x, nullptr, rows, on_device)) return rc;
    if (int rc = mlp_fwd(m, rows)) return rc;
    QSIM_CUDA(cudaMemcpyAsync(y, m->y, sizeof(float) * rows, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                              m->stream));
    QSIM_CUDA(cudaStreamSynchronize(m->stream));
    return SIM_OK;
}

int sim_mlp_loss_grad(qsim_mlp *m, const float *x, const float *t, int64_t rows, int on_device, float *loss,
                      float *grad_host)
{
    if (!m || !x || !t || rows < 1) return fail(SIM_EINVAL, "sim_mlp_loss_grad: bad arguments");
    if (int rc = mlp_load_xy(m, x, t, rows, on_device)) return rc;
    if (int rc = mlp_fwd(m, rows)) return rc;
    if (int rc = mlp_bwd(m, rows)) return rc;
    if (loss) QSIM_CUDA(cudaMemcpyAsync(loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->stream));
    if (grad_host)
        QSIM_CUDA(cudaMemcpyAsync(grad_host, m->grad, sizeof(float) * m->off.total, cudaMemcpyDeviceToHost, m->stream));
    QSIM_CUDA(cudaStreamSynchronize(m->stream));
    return SIM_OK;
}

int sim_mlp_train(qsim_mlp *m, const float *x, const float *t, int64_t rows, int steps, float lr, int on_device,
                  float *final_loss)
{
    if (!m || !x || !t || rows < 1 || steps < 0) return fail(SIM_EINVAL, "sim_mlp_train: bad arguments");
    if (int rc = mlp_load_xy(m, x, t, rows, on_device)) return rc;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int s = 0; s < steps; ++s) {
        if (int rc = mlp_fwd(m, rows)) return rc;
        if (int rc = mlp_bwd(m, rows)) return rc;
        m->t += 1;
        const float c1 = 1.f - powf(b1, (float)m->t), c2 = 1.f - powf(b2, (float)m->t);
        k_adam<<<blocks_for(m->off.total, 256), 256, 0, m->stream>>>(m->theta, m->grad, m->m, m->v, m->off.total, lr,
                                                                    b1, b2, eps, c1, c2);
        QSIM_CUDA(cudaGetLastError());
    }
    if (final_loss) {
        if (int rc = mlp_fwd(m, rows)) return rc;
        k_mse<<<1, 256, 0, m->stream>>>(m->y, m->tgt, rows, m->loss);
        QSIM_CUDA(cudaMemcpyAsync(final_loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->stream));
    }
    QSIM_CUDA(cudaStreamSynchronize(m->stream));
    return SIM_OK;
}

}  // extern "C"
