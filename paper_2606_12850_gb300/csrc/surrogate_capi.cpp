// C ABI of the seismogram surrogate (include/surrogate.h): the model owns its parameters,
// Adam state, activations and scratch on one GPU and orders the kernel launches of the
// forward pass, the backward pass and the optimiser step.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "sem.h"
#include "surrogate.h"
#include "surrogate_internal.h"

using sgk::bf16;

struct sg_model {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int in_dim = 0, hidden = 0, c0 = 0, l0 = 0, nstages = 0, max_batch = 0;
  int contract = 0;  // output linear in the last `contract` inputs (0: the last stage is the output)
  std::vector<int> cin, cout, up, lin, lout;
  int out_c = 0, out_l = 0;
  size_t oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, oW3 = 0, ob3 = 0, P = 0;
  std::vector<size_t> oC, oc;
  float *d_p = nullptr, *d_g = nullptr, *d_m = nullptr, *d_v = nullptr;
  bf16* d_pb = nullptr;
  float *d_a1 = nullptr, *d_h1 = nullptr, *d_a2 = nullptr, *d_h2 = nullptr, *d_a3 = nullptr, *d_z0 = nullptr;
  std::vector<float*> d_pre, d_out;
  float *d_dA = nullptr, *d_dB = nullptr;
  float* d_y = nullptr;  // network output [max_batch][out_c][out_l] when contract > 0
  float* d_ws = nullptr;
  double* d_partials = nullptr;
  int* d_err = nullptr;  // set by a tensor-core product whose bounded wait ran out
  bf16* d_pack = nullptr;  // the convolutions' weights packed for the tcgen05 kernel
  float* d_red = nullptr;  // per-slice sums of the bias gradients
  sgk::Products prod;    // product kernel (SG_OPT_PRODUCT) and d_err
  long long step = 0;
  size_t dev_bytes = 0;
  std::vector<void*> allocs;
  std::string err;
};

namespace {

std::string g_sg_err;
constexpr size_t kRedFloats = 8192;  // bias-gradient slice sums: up to 8192 / channels slices

int sg_fail(sg_model* m, int code, const std::string& msg) {
  if (m)
    m->err = msg;
  else
    g_sg_err = msg;
  return code;
}

#define SG_CUDA(m, call)                                                                     \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) return sg_fail((m), SEM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define SG_LAUNCH(m, call)                                                                   \
  do {                                                                                       \
    int r_ = (call);                                                                         \
    if (r_ != 0)                                                                             \
      return sg_fail((m), SEM_ECUDA,                                                         \
                     std::string(#call) + ": " + cudaGetErrorString(static_cast<cudaError_t>(r_))); \
  } while (0)

template <typename T>
int sg_alloc(sg_model* m, T** p, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
  if (e != cudaSuccess) return sg_fail(m, SEM_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  m->allocs.push_back(q);
  m->dev_bytes += count * sizeof(T);
  *p = static_cast<T*>(q);
  return SG_OK;
}

// After a stream synchronisation: a product kernel that gave up waiting for the tensor cores
// left d_err set; report it (and clear it for the next call).
int check_products(sg_model* m, const char* where) {
  int h = 0;
  SG_CUDA(m, cudaMemcpy(&h, m->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (h == 0) return SG_OK;
  SG_CUDA(m, cudaMemset(m->d_err, 0, sizeof(int)));
  return sg_fail(m, SEM_ETIMEOUT, std::string(where) + ": a tensor-core product timed out waiting for its MMAs");
}

int forward_chunk(sg_model* m, int b, const float* x, float* y_last) {
  cudaStream_t s = m->stream;
  SG_LAUNCH(m, sgk::linear_forward(b, m->in_dim, m->hidden, x, m->d_pb + m->oW1, m->d_p + m->ob1, m->d_a1, m->d_h1,
                                   true, m->prod, s));
  SG_LAUNCH(m, sgk::linear_forward(b, m->hidden, m->hidden, m->d_h1, m->d_pb + m->oW2, m->d_p + m->ob2, m->d_a2,
                                   m->d_h2, true, m->prod, s));
  SG_LAUNCH(m, sgk::linear_forward(b, m->hidden, m->c0 * m->l0, m->d_h2, m->d_pb + m->oW3, m->d_p + m->ob3, m->d_a3,
                                   m->d_z0, true, m->prod, s));
  const float* in = m->d_z0;
  const int last = m->nstages - 1;
  for (int st = 0; st < m->nstages; ++st) {
    float* pre = (st == last && y_last && !m->contract) ? y_last : m->d_pre[st];
    float* out = st == last ? nullptr : m->d_out[st];
    SG_LAUNCH(m, sgk::conv_forward(b, m->cin[st], m->cout[st], m->lin[st], m->up[st], in, m->d_pb + m->oC[st],
                                   m->d_p + m->oc[st], pre, out, m->prod, s));
    in = out;
  }
  if (m->contract)
    SG_LAUNCH(m, sgk::contract_forward(b, m->contract, m->out_c, m->out_l, m->in_dim, x, m->d_pre[last],
                                       y_last ? y_last : m->d_y, s));
  return SG_OK;
}

}  // namespace

extern "C" {

int sg_create(sg_model** out, int device, void* stream, int in_dim, int hidden, int c0, int l0, int nstages,
              const int32_t* stage_cout, const int32_t* stage_up, int contract, int max_batch) {
  if (!out) return sg_fail(nullptr, SEM_EINVAL, "sg_create: NULL output");
  *out = nullptr;
  if (in_dim < 1 || hidden < 1 || c0 < 1 || l0 < 1 || nstages < 1 || nstages > SG_MAX_STAGES || !stage_cout ||
      !stage_up || max_batch < 1)
    return sg_fail(nullptr, SEM_EINVAL, "sg_create: bad sizes");
  sg_model* m = new sg_model();
  m->device = device;
  m->in_dim = in_dim;
  m->hidden = hidden;
  m->c0 = c0;
  m->l0 = l0;
  m->nstages = nstages;
  m->max_batch = max_batch;
  int c = c0, l = l0;
  for (int st = 0; st < nstages; ++st) {
    if (stage_cout[st] < 1 || (stage_up[st] != 1 && stage_up[st] != 2)) {
      delete m;
      return sg_fail(nullptr, SEM_EINVAL, "sg_create: stage channels must be >= 1 and upsampling 1 or 2");
    }
    m->cin.push_back(c);
    m->cout.push_back(stage_cout[st]);
    m->up.push_back(stage_up[st]);
    m->lin.push_back(l);
    l *= stage_up[st];
    m->lout.push_back(l);
    c = stage_cout[st];
  }
  if (contract < 0 || contract > in_dim || (contract > 0 && c % contract != 0)) {
    delete m;
    return sg_fail(nullptr, SEM_EINVAL, "sg_create: contract must divide the last stage's channels and be <= in_dim");
  }
  // the products' index maps divide sample indices (up to max_batch x length) by a float
  // reciprocal, exact below 2^24
  if (static_cast<long long>(max_batch) * l >= (1LL << 24)) {
    delete m;
    return sg_fail(nullptr, SEM_EINVAL, "sg_create: max_batch x output length must be below 2^24");
  }
  m->contract = contract;
  m->out_c = contract ? c / contract : c;
  m->out_l = l;
  size_t o = 0;
  m->oW1 = o; o += static_cast<size_t>(hidden) * in_dim;
  m->ob1 = o; o += hidden;
  m->oW2 = o; o += static_cast<size_t>(hidden) * hidden;
  m->ob2 = o; o += hidden;
  m->oW3 = o; o += static_cast<size_t>(c0) * l0 * hidden;
  m->ob3 = o; o += static_cast<size_t>(c0) * l0;
  for (int st = 0; st < nstages; ++st) {
    m->oC.push_back(o); o += static_cast<size_t>(m->cout[st]) * m->cin[st] * 3;
    m->oc.push_back(o); o += m->cout[st];
  }
  m->P = o;
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) {
    if (stream) {
      m->stream = static_cast<cudaStream_t>(stream);
    } else {
      e = cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking);
      m->own_stream = e == cudaSuccess;
    }
  }
  if (e != cudaSuccess) {
    delete m;
    return sg_fail(nullptr, SEM_ECUDA, std::string("sg_create: ") + cudaGetErrorString(e));
  }
  const size_t B = max_batch;
  size_t act = std::max<size_t>(static_cast<size_t>(c0) * l0, hidden);
  for (int st = 0; st < nstages; ++st) {
    act = std::max(act, static_cast<size_t>(m->cout[st]) * m->lout[st]);
    act = std::max(act, static_cast<size_t>(m->cin[st]) * m->lin[st]);
  }
  size_t ws = 0;
  ws = std::max(ws, sgk::splitk_floats(hidden, in_dim, max_batch));
  ws = std::max(ws, sgk::splitk_floats(hidden, hidden, max_batch));
  ws = std::max(ws, sgk::splitk_floats(c0 * l0, hidden, max_batch));
  ws = std::max(ws, sgk::splitk_floats(max_batch, hidden, c0 * l0));  // backward data of the dense layers
  ws = std::max(ws, sgk::splitk_floats(max_batch, hidden, hidden));
  for (int st = 0; st < nstages; ++st)
    ws = std::max(ws, sgk::splitk_floats(m->cout[st], m->cin[st] * 3, max_batch * m->lout[st]));
  size_t pack = 0;
  for (int st = 0; st < nstages; ++st) pack = std::max(pack, sgk::conv_pack_bytes(m->cin[st], m->cout[st]));
  int r = SG_OK;
  if ((r = sg_alloc(m, &m->d_p, m->P)) || (r = sg_alloc(m, &m->d_g, m->P)) || (r = sg_alloc(m, &m->d_m, m->P)) ||
      (r = sg_alloc(m, &m->d_v, m->P)) || (r = sg_alloc(m, &m->d_pb, m->P)) ||
      (r = sg_alloc(m, &m->d_a1, B * hidden)) || (r = sg_alloc(m, &m->d_h1, B * hidden)) ||
      (r = sg_alloc(m, &m->d_a2, B * hidden)) || (r = sg_alloc(m, &m->d_h2, B * hidden)) ||
      (r = sg_alloc(m, &m->d_a3, B * c0 * l0)) || (r = sg_alloc(m, &m->d_z0, B * c0 * l0)) ||
      (r = sg_alloc(m, &m->d_dA, B * act)) || (r = sg_alloc(m, &m->d_dB, B * act)) ||
      (r = sg_alloc(m, &m->d_ws, ws)) || (r = sg_alloc(m, &m->d_partials, sgk::kLossBlocks)) ||
      (r = sg_alloc(m, &m->d_err, 1)) || (r = sg_alloc(m, &m->d_pack, pack / sizeof(bf16))) ||
      (r = sg_alloc(m, &m->d_red, kRedFloats)) ||
      (r = sg_alloc(m, &m->d_y, contract ? B * m->out_c * m->out_l : 0))) {
    std::string msg = m->err;
    sg_destroy(m);
    return sg_fail(nullptr, r, msg);
  }
  m->d_pre.assign(nstages, nullptr);
  m->d_out.assign(nstages, nullptr);
  for (int st = 0; st < nstages && r == SG_OK; ++st) {
    const size_t n = B * m->cout[st] * m->lout[st];
    r = sg_alloc(m, &m->d_pre[st], n);
    if (r == SG_OK && st + 1 < nstages) r = sg_alloc(m, &m->d_out[st], n);
  }
  if (r == SG_OK) {
    const size_t bytes = m->P * sizeof(float);
    cudaError_t z = cudaSuccess;
    float* zero[4] = {m->d_p, m->d_g, m->d_m, m->d_v};
    for (float* q : zero)
      if (z == cudaSuccess) z = cudaMemsetAsync(q, 0, bytes, m->stream);
    if (z == cudaSuccess) z = cudaMemsetAsync(m->d_pb, 0, m->P * sizeof(bf16), m->stream);
    if (z == cudaSuccess) z = cudaMemsetAsync(m->d_err, 0, sizeof(int), m->stream);
    if (z == cudaSuccess) z = cudaStreamSynchronize(m->stream);
    if (z != cudaSuccess) r = sg_fail(m, SEM_ECUDA, std::string("sg_create: ") + cudaGetErrorString(z));
  }
  if (r != SG_OK) {
    std::string msg = m->err;
    sg_destroy(m);
    return sg_fail(nullptr, r, msg);
  }
  m->prod.err = m->d_err;
  m->prod.pack = m->d_pack;
  m->prod.pack_bytes = pack;
  m->prod.red = m->d_red;
  m->prod.red_floats = kRedFloats;
  m->prod.ws_floats = ws;
  *out = m;
  return SG_OK;
}

int sg_destroy(sg_model* m) {
  if (!m) return SG_OK;
  cudaSetDevice(m->device);
  if (m->stream) cudaStreamSynchronize(m->stream);
  for (void* p : m->allocs) cudaFree(p);
  if (m->own_stream && m->stream) cudaStreamDestroy(m->stream);
  delete m;
  return SG_OK;
}

int sg_info(sg_model* m, int64_t* out) {
  if (!m || !out) return sg_fail(m, SEM_EINVAL, "sg_info: bad arguments");
  out[0] = static_cast<int64_t>(m->P);
  out[1] = m->out_c;
  out[2] = m->out_l;
  out[3] = static_cast<int64_t>(m->dev_bytes);
  return SG_OK;
}

int sg_set_params(sg_model* m, const float* params) {
  if (!m || !params) return sg_fail(m, SEM_EINVAL, "sg_set_params: bad arguments");
  for (size_t i = 0; i < m->P; ++i)
    if (!std::isfinite(params[i])) return sg_fail(m, SEM_EINVAL, "sg_set_params: non-finite parameter");
  SG_CUDA(m, cudaSetDevice(m->device));
  SG_CUDA(m, cudaMemcpyAsync(m->d_p, params, m->P * sizeof(float), cudaMemcpyHostToDevice, m->stream));
  SG_CUDA(m, cudaMemsetAsync(m->d_m, 0, m->P * sizeof(float), m->stream));
  SG_CUDA(m, cudaMemsetAsync(m->d_v, 0, m->P * sizeof(float), m->stream));
  SG_LAUNCH(m, sgk::to_bf16(m->P, m->d_p, m->d_pb, m->stream));
  SG_CUDA(m, cudaStreamSynchronize(m->stream));
  m->step = 0;
  return SG_OK;
}

int sg_get_params(sg_model* m, float* params) {
  if (!m || !params) return sg_fail(m, SEM_EINVAL, "sg_get_params: bad arguments");
  SG_CUDA(m, cudaSetDevice(m->device));
  SG_CUDA(m, cudaMemcpyAsync(params, m->d_p, m->P * sizeof(float), cudaMemcpyDeviceToHost, m->stream));
  SG_CUDA(m, cudaStreamSynchronize(m->stream));
  return SG_OK;
}

int sg_get_grads(sg_model* m, float* grads) {
  if (!m || !grads) return sg_fail(m, SEM_EINVAL, "sg_get_grads: bad arguments");
  SG_CUDA(m, cudaSetDevice(m->device));
  SG_CUDA(m, cudaMemcpyAsync(grads, m->d_g, m->P * sizeof(float), cudaMemcpyDeviceToHost, m->stream));
  SG_CUDA(m, cudaStreamSynchronize(m->stream));
  return SG_OK;
}

int sg_forward(sg_model* m, int batch, const float* x, float* y) {
  if (!m) return sg_fail(nullptr, SEM_EINVAL, "null model");
  if (batch < 0 || (batch > 0 && (!x || !y))) return sg_fail(m, SEM_EINVAL, "sg_forward: bad arguments");
  SG_CUDA(m, cudaSetDevice(m->device));
  const size_t per_out = static_cast<size_t>(m->out_c) * m->out_l;
  for (int b0 = 0; b0 < batch; b0 += m->max_batch) {
    const int b = std::min(m->max_batch, batch - b0);
    int r = forward_chunk(m, b, x + static_cast<size_t>(b0) * m->in_dim, y + b0 * per_out);
    if (r) return r;
  }
  return SG_OK;
}

int sg_loss_grad(sg_model* m, int b, const float* x, const float* target, double* loss) {
  if (!m) return sg_fail(nullptr, SEM_EINVAL, "null model");
  if (b < 1 || b > m->max_batch || !x || !target || !loss) return sg_fail(m, SEM_EINVAL, "sg_loss_grad: bad arguments");
  SG_CUDA(m, cudaSetDevice(m->device));
  cudaStream_t s = m->stream;
  int r = forward_chunk(m, b, x, nullptr);
  if (r) return r;
  const int last = m->nstages - 1;
  const size_t n = static_cast<size_t>(b) * m->out_c * m->out_l;
  float* cur = m->d_dA;
  float* other = m->d_dB;
  SG_LAUNCH(m, sgk::mse_grad(n, m->contract ? m->d_y : m->d_pre[last], target, cur, m->d_partials, s));
  if (m->contract) {
    SG_LAUNCH(m, sgk::contract_backward(b, m->contract, m->out_c, m->out_l, m->in_dim, x, cur, other, s));
    std::swap(cur, other);
  }
  for (int st = last; st >= 0; --st) {
    if (st != last)
      SG_LAUNCH(m, sgk::gelu_backward(static_cast<size_t>(b) * m->cout[st] * m->lout[st], m->d_pre[st], cur, s));
    const float* input = st == 0 ? m->d_z0 : m->d_out[st - 1];
    SG_LAUNCH(m, sgk::conv_backward_weight(b, m->cin[st], m->cout[st], m->lin[st], m->up[st], cur, input,
                                           m->d_g + m->oC[st], m->d_g + m->oc[st], m->d_ws, m->prod, s));
    SG_LAUNCH(m, sgk::conv_backward_data(b, m->cin[st], m->cout[st], m->lin[st], m->up[st], cur, m->d_pb + m->oC[st],
                                         other, m->prod, s));
    std::swap(cur, other);
  }
  const int n3 = m->c0 * m->l0;
  SG_LAUNCH(m, sgk::gelu_backward(static_cast<size_t>(b) * n3, m->d_a3, cur, s));
  SG_LAUNCH(m, sgk::linear_backward_weight(b, m->hidden, n3, cur, m->d_h2, m->d_g + m->oW3, m->d_g + m->ob3, m->d_ws,
                                           m->prod, s));
  SG_LAUNCH(m, sgk::linear_backward_data(b, m->hidden, n3, cur, m->d_pb + m->oW3, other, m->d_ws, m->prod, s));
  std::swap(cur, other);
  SG_LAUNCH(m, sgk::gelu_backward(static_cast<size_t>(b) * m->hidden, m->d_a2, cur, s));
  SG_LAUNCH(m, sgk::linear_backward_weight(b, m->hidden, m->hidden, cur, m->d_h1, m->d_g + m->oW2, m->d_g + m->ob2,
                                           m->d_ws, m->prod, s));
  SG_LAUNCH(m, sgk::linear_backward_data(b, m->hidden, m->hidden, cur, m->d_pb + m->oW2, other, m->d_ws, m->prod, s));
  std::swap(cur, other);
  SG_LAUNCH(m, sgk::gelu_backward(static_cast<size_t>(b) * m->hidden, m->d_a1, cur, s));
  SG_LAUNCH(m, sgk::linear_backward_weight(b, m->in_dim, m->hidden, cur, x, m->d_g + m->oW1, m->d_g + m->ob1, m->d_ws,
                                           m->prod, s));
  std::vector<double> part(sgk::kLossBlocks);
  SG_CUDA(m, cudaMemcpyAsync(part.data(), m->d_partials, part.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  SG_CUDA(m, cudaStreamSynchronize(s));
  if (int e = check_products(m, "sg_loss_grad")) return e;
  double sum = 0.0;
  for (double v : part) sum += v;
  *loss = sum / static_cast<double>(n);
  return SG_OK;
}

int sg_adam_step(sg_model* m, float lr, float beta1, float beta2, float eps) {
  if (!m) return sg_fail(nullptr, SEM_EINVAL, "null model");
  if (!(lr >= 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps >= 0.f))
    return sg_fail(m, SEM_EINVAL, "sg_adam_step: bad hyper-parameters");
  SG_CUDA(m, cudaSetDevice(m->device));
  ++m->step;
  const double c1 = 1.0 - std::pow(static_cast<double>(beta1), static_cast<double>(m->step));
  const double c2 = 1.0 - std::pow(static_cast<double>(beta2), static_cast<double>(m->step));
  SG_LAUNCH(m, sgk::adam_update(m->P, m->d_p, m->d_g, m->d_m, m->d_v, m->d_pb, lr, beta1, beta2, eps,
                                static_cast<float>(1.0 / c1), static_cast<float>(1.0 / c2), m->stream));
  return SG_OK;
}

int sg_sync(sg_model* m) {
  if (!m) return sg_fail(nullptr, SEM_EINVAL, "null model");
  SG_CUDA(m, cudaSetDevice(m->device));
  SG_CUDA(m, cudaStreamSynchronize(m->stream));
  return check_products(m, "sg_sync");
}

int sg_set_option(sg_model* m, int option, int value) {
  if (!m) return sg_fail(nullptr, SEM_EINVAL, "null model");
  if ((option != SG_OPT_PRODUCT && option != SG_OPT_STALL_TEST) || (value != 0 && value != 1))
    return sg_fail(m, SEM_EINVAL, "sg_set_option: unknown option or value");
  SG_CUDA(m, cudaSetDevice(m->device));
  SG_CUDA(m, cudaStreamSynchronize(m->stream));
  (option == SG_OPT_PRODUCT ? m->prod.kind : m->prod.stall_test) = value;
  return SG_OK;
}

int sg_get_option(sg_model* m, int option, int* value) {
  if (!m || !value || (option != SG_OPT_PRODUCT && option != SG_OPT_STALL_TEST))
    return sg_fail(m, SEM_EINVAL, "sg_get_option: bad arguments");
  *value = option == SG_OPT_PRODUCT ? m->prod.kind : m->prod.stall_test;
  return SG_OK;
}

const char* sg_last_error(const sg_model* m) { return m ? m->err.c_str() : g_sg_err.c_str(); }

}  // extern "C"
