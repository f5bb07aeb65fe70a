// Training and inference kernels of the MLP cost model that picks a map and
// block size (not part of the paper): y = W3 relu(W2 relu(W1 x + b1) + b2) + b3,
// mean-squared-error loss, Adam (Kingma and Ba, 2015).  Every reduction runs
// in a fixed order, so results do not depend on scheduling.
#include <cuda_runtime.h>

#include "../../include/tri.h"

namespace {

// out[b][o] = sum_i W[o][i] act(in[b][i]) + bias[o], act = relu when in_relu
__global__ void dense_fwd_kernel(const float *__restrict__ in, int in_relu, const float *__restrict__ W,
                                 const float *__restrict__ bias, float *__restrict__ out, uint32_t B, uint32_t I,
                                 uint32_t O)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= B * O) return;
    const uint32_t b = t / O, o = t - b * O;
    const float *x = in + (size_t)b * I, *w = W + (size_t)o * I;
    float s = bias[o];
    for (uint32_t i = 0; i < I; ++i) {
        const float v = in_relu ? fmaxf(x[i], 0.0f) : x[i];
        s = fmaf(w[i], v, s);
    }
    out[(size_t)b * O + o] = s;
}

// r = pred - y; g_out = (2/B) r; loss = mean r^2 (one block, fixed order)
__global__ void loss_kernel(const float *__restrict__ pred, const float *__restrict__ y, uint32_t B,
                            float *__restrict__ g_out, float *__restrict__ loss)
{
    __shared__ float part[256];
    float s = 0.0f;
    for (uint32_t b = threadIdx.x; b < B; b += blockDim.x) {
        const float r = pred[b] - y[b];
        g_out[b] = 2.0f * r / (float)B;
        s = fmaf(r, r, s);
    }
    part[threadIdx.x] = s;
    __syncthreads();
    for (uint32_t w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = part[0] / (float)B;
}

// gprev[b][i] = (sum_o gnext[b][o] W[o][i]) * (zprev[b][i] > 0)
__global__ void backprop_kernel(const float *__restrict__ gnext, const float *__restrict__ W,
                                const float *__restrict__ zprev, float *__restrict__ gprev, uint32_t B, uint32_t I,
                                uint32_t O)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= B * I) return;
    const uint32_t b = t / I, i = t - b * I;
    float s = 0.0f;
    for (uint32_t o = 0; o < O; ++o) s = fmaf(gnext[(size_t)b * O + o], W[(size_t)o * I + i], s);
    gprev[t] = zprev[t] > 0.0f ? s : 0.0f;
}

// gW[o][i] = sum_b g[b][o] act(a[b][i]); gbias[o] = sum_b g[b][o]
__global__ void wgrad_kernel(const float *__restrict__ g, const float *__restrict__ a, int a_relu,
                             float *__restrict__ gW, float *__restrict__ gbias, uint32_t B, uint32_t I, uint32_t O)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= O * (I + 1)) return;
    const uint32_t o = t / (I + 1), i = t - o * (I + 1);
    float s = 0.0f;
    if (i < I) {
        for (uint32_t b = 0; b < B; ++b) {
            const float v = a[(size_t)b * I + i];
            s = fmaf(g[(size_t)b * O + o], a_relu ? fmaxf(v, 0.0f) : v, s);
        }
        gW[(size_t)o * I + i] = s;
    } else {
        for (uint32_t b = 0; b < B; ++b) s += g[(size_t)b * O + o];
        gbias[o] = s;
    }
}

__global__ void adam_kernel(float *__restrict__ theta, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, uint32_t np, float lr, float b1, float b2, float eps, float c1,
                            float c2)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= np) return;
    const float gt = g[t];
    const float mt = b1 * m[t] + (1.0f - b1) * gt;
    const float vt = b2 * v[t] + (1.0f - b2) * gt * gt;
    m[t] = mt;
    v[t] = vt;
    theta[t] -= lr * (mt / c1) / (sqrtf(vt / c2) + eps);
}

__global__ void argmin_kernel(const float *__restrict__ pred, uint32_t B, uint32_t *__restrict__ best)
{
    __shared__ float bv[256];
    __shared__ uint32_t bi[256];
    float v = __int_as_float(0x7f800000);
    uint32_t k = 0xFFFFFFFFu;
    for (uint32_t b = threadIdx.x; b < B; b += blockDim.x)
        if (pred[b] < v) {
            v = pred[b];
            k = b;
        }
    bv[threadIdx.x] = v;
    bi[threadIdx.x] = k;
    __syncthreads();
    for (uint32_t w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            const float ov = bv[threadIdx.x + w];
            const uint32_t ok = bi[threadIdx.x + w];
            if (ov < bv[threadIdx.x] || (ov == bv[threadIdx.x] && ok < bi[threadIdx.x])) {
                bv[threadIdx.x] = ov;
                bi[threadIdx.x] = ok;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *best = bi[0] == 0xFFFFFFFFu ? 0 : bi[0];
}

inline unsigned nblk(size_t work) { return (unsigned)((work + 255) / 256); }

struct Layout {
    const float *W1, *b1, *W2, *b2, *W3, *b3;
};

Layout layout(const float *theta, uint32_t F, uint32_t H1, uint32_t H2)
{
    Layout L;
    L.W1 = theta;
    L.b1 = L.W1 + (size_t)H1 * F;
    L.W2 = L.b1 + H1;
    L.b2 = L.W2 + (size_t)H2 * H1;
    L.W3 = L.b2 + H2;
    L.b3 = L.W3 + H2;
    return L;
}

bool shapes_ok(uint32_t B, uint32_t F, uint32_t H1, uint32_t H2)
{
    return B > 0 && F > 0 && F <= 64 && H1 > 0 && H1 <= 128 && H2 > 0 && H2 <= 128;
}

// workspace: z1 [B][H1], z2 [B][H2], pred [B], g_out [B], g_z2 [B][H2], g_z1 [B][H1]
size_t ws_floats(uint32_t B, uint32_t H1, uint32_t H2) { return (size_t)B * (2 * H1 + 2 * H2 + 2); }

int forward(const float *theta, const float *X, uint32_t B, uint32_t F, uint32_t H1, uint32_t H2, float *pred,
            float *ws, cudaStream_t s)
{
    const Layout L = layout(theta, F, H1, H2);
    float *z1 = ws, *z2 = z1 + (size_t)B * H1;
    dense_fwd_kernel<<<nblk((size_t)B * H1), 256, 0, s>>>(X, 0, L.W1, L.b1, z1, B, F, H1);
    dense_fwd_kernel<<<nblk((size_t)B * H2), 256, 0, s>>>(z1, 1, L.W2, L.b2, z2, B, H1, H2);
    dense_fwd_kernel<<<nblk(B), 256, 0, s>>>(z2, 1, L.W3, L.b3, pred, B, H2, 1);
    return cudaGetLastError() == cudaSuccess ? TRI_OK : TRI_ECUDA;
}

}  // namespace

extern "C" int tri_mlp_workspace_size(uint32_t B, uint32_t H1, uint32_t H2, size_t *bytes)
{
    if (!bytes) return TRI_EINVAL;
    *bytes = ws_floats(B, H1, H2) * sizeof(float);
    return TRI_OK;
}

extern "C" int tri_mlp_forward(const float *theta, const float *X, uint32_t B, uint32_t F, uint32_t H1, uint32_t H2,
                               float *pred, void *workspace, size_t ws_bytes, void *stream)
{
    if (!theta || !X || !pred || !workspace || !shapes_ok(B, F, H1, H2)) return TRI_EINVAL;
    if (ws_bytes < ws_floats(B, H1, H2) * sizeof(float)) return TRI_ENOSPACE;
    return forward(theta, X, B, F, H1, H2, pred, (float *)workspace, (cudaStream_t)stream);
}

extern "C" int tri_mlp_grad(const float *theta, const float *X, const float *y, uint32_t B, uint32_t F, uint32_t H1,
                            uint32_t H2, float *loss, float *grad, void *workspace, size_t ws_bytes, void *stream)
{
    if (!theta || !X || !y || !loss || !grad || !workspace || !shapes_ok(B, F, H1, H2)) return TRI_EINVAL;
    if (ws_bytes < ws_floats(B, H1, H2) * sizeof(float)) return TRI_ENOSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    float *ws = (float *)workspace;
    float *z1 = ws, *z2 = z1 + (size_t)B * H1, *pred = z2 + (size_t)B * H2, *g_out = pred + B;
    float *g_z2 = g_out + B, *g_z1 = g_z2 + (size_t)B * H2;
    int st = forward(theta, X, B, F, H1, H2, pred, ws, s);
    if (st != TRI_OK) return st;
    const Layout L = layout(theta, F, H1, H2);
    float *gW1 = grad, *gb1 = gW1 + (size_t)H1 * F, *gW2 = gb1 + H1, *gb2 = gW2 + (size_t)H2 * H1;
    float *gW3 = gb2 + H2, *gb3 = gW3 + H2;
    loss_kernel<<<1, 256, 0, s>>>(pred, y, B, g_out, loss);
    wgrad_kernel<<<nblk(H2 + 1), 256, 0, s>>>(g_out, z2, 1, gW3, gb3, B, H2, 1);
    backprop_kernel<<<nblk((size_t)B * H2), 256, 0, s>>>(g_out, L.W3, z2, g_z2, B, H2, 1);
    wgrad_kernel<<<nblk((size_t)H2 * (H1 + 1)), 256, 0, s>>>(g_z2, z1, 1, gW2, gb2, B, H1, H2);
    backprop_kernel<<<nblk((size_t)B * H1), 256, 0, s>>>(g_z2, L.W2, z1, g_z1, B, H1, H2);
    wgrad_kernel<<<nblk((size_t)H1 * (F + 1)), 256, 0, s>>>(g_z1, X, 0, gW1, gb1, B, F, H1);
    return cudaGetLastError() == cudaSuccess ? TRI_OK : TRI_ECUDA;
}

extern "C" int tri_mlp_adam(float *theta, const float *grad, float *m, float *v, uint32_t nparams, uint32_t t,
                            float lr, float beta1, float beta2, float eps, void *stream)
{
    if (!theta || !grad || !m || !v || nparams == 0 || t == 0) return TRI_EINVAL;
    const float c1 = 1.0f - powf(beta1, (float)t), c2 = 1.0f - powf(beta2, (float)t);
    adam_kernel<<<nblk(nparams), 256, 0, (cudaStream_t)stream>>>(theta, grad, m, v, nparams, lr, beta1, beta2, eps,
                                                                  c1, c2);
    return cudaGetLastError() == cudaSuccess ? TRI_OK : TRI_ECUDA;
}

extern "C" int tri_mlp_argmin(const float *theta, const float *X, uint32_t B, uint32_t F, uint32_t H1, uint32_t H2,
                              uint32_t *best, void *workspace, size_t ws_bytes, void *stream)
{
    if (!theta || !X || !best || !workspace || !shapes_ok(B, F, H1, H2)) return TRI_EINVAL;
    if (ws_bytes < ws_floats(B, H1, H2) * sizeof(float)) return TRI_ENOSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    float *ws = (float *)workspace;
    float *pred = ws + (size_t)B * (H1 + H2);
    int st = forward(theta, X, B, F, H1, H2, pred, ws, s);
    if (st != TRI_OK) return st;
    argmin_kernel<<<1, 256, 0, s>>>(pred, B, best);
    return cudaGetLastError() == cudaSuccess ? TRI_OK : TRI_ECUDA;
}
