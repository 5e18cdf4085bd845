// Host side of the learned warm start (declared in include/ptycho.h):
// parameters, buffers, the forward / backward launch sequence, AdamW, and the
// stitching of predicted patches into a reconstruction's initial object.
// Included by ptycho_api.cu (uses the context internals).

struct ptycho_net {
  cudaStream_t st = nullptr;
  cudaStream_t st_side = nullptr;  // bias gradients and weight split sums beside the main chain
  cudaEvent_t ev_fork1 = nullptr, ev_fork2 = nullptr, ev_join = nullptr;
  int max_batch = 0;
  long long n_params = 0, n_w = 0;
  long long w_off[NET_LAYERS], b_off[NET_LAYERS], wb_off[NET_LAYERS];
  float* params = nullptr;   // FP32 master
  float* grads = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  __nv_bfloat16* wb = nullptr;  // BF16 weights [co][ci][9]
  __nv_bfloat16* wt = nullptr;  // the same, tap-major [co][9][ci] (inference path)
  bool wt_valid = false;        // wt matches wb
  unsigned char* is_w = nullptr;
  int* wb_index = nullptr;
  int* wt_index = nullptr;      // position of each weight in wt
  bool f32 = false;             // FP32 activations (verification mode)
  bool tc = true;               // forward convolutions on the tensor cores (BF16 mode)
  int* err_flag = nullptr;      // set by a bounded device wait that gave up
  float* tc_part = nullptr;     // split-K partial tiles of the tensor-core forward
  size_t tc_part_n = 0;
  double* bpart = nullptr;      // bias-gradient slice sums [slice][channel]
  float* bd_part = nullptr;     // split-K partial tiles of the tensor-core data gradient
  size_t bd_part_n = 0;
  size_t wpart_n = 0;           // capacity of wpart (floats)
  void* x = nullptr;            // input [B][1][128][128]
  void* act[NET_LAYERS] = {};   // layers 0..10 (BF16, or FP32 in verification mode)
  float* out = nullptr;         // layer 11 output [B][2][64][64] (FP32)
  float* delta[2] = {nullptr, nullptr};
  float* wpart = nullptr;
  double* lpart = nullptr;
  long long adam_t = 0;
  std::string err;
};

constexpr int NET_BPART = 4096;  // capacity of the bias-gradient slice sums (doubles)

namespace {

thread_local std::string g_net_error;

int nfail(ptycho_net* n, int code, const char* fmt, ...) {
  char t[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(t, sizeof t, fmt, ap);
  va_end(ap);
  if (n) n->err = t;
  else g_net_error = t;
  return code;
}

template <typename T>
int nalloc(ptycho_net* n, T** p, size_t count) {
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T) + 16);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return nfail(n, PTYCHO_ERR_OOM, "cudaMalloc of %zu bytes: %s", count * sizeof(T), cudaGetErrorString(e));
  }
  return 0;
}

size_t act_size(int l, int B) {
  const NetLayer L = net_layer(l);
  return (size_t)B * L.co * L.hout * L.wout;
}

int net_check(ptycho_net* n, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return nfail(n, PTYCHO_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
  return 0;
}

ConvArgs conv_args(ptycho_net* n, int l, int B) {
  const NetLayer L = net_layer(l);
  ConvArgs a{};
  a.in = l == 0 ? n->x : n->act[l - 1];
  a.w = n->wb + n->wb_off[l];
  a.b = n->params + n->b_off[l];
  a.B = B;
  a.ci = L.ci;
  a.co = L.co;
  a.hin = L.hin;
  a.win = L.win;
  a.hout = L.hout;
  a.wout = L.wout;
  a.stride = L.stride;
  a.up = L.up;
  a.relu = L.relu;
  return a;
}

template <typename TA>
int net_forward_t(ptycho_net* n, int B) {
  for (int l = 0; l < NET_LAYERS; ++l) {
    const NetLayer L = net_layer(l);
    ConvArgs a = conv_args(n, l, B);
    const dim3 g((unsigned)(((long long)B * L.hout * L.wout + CV_NT - 1) / CV_NT), (unsigned)((L.co + CV_CO - 1) / CV_CO));
    if (l == NET_LAYERS - 1) {
      a.out = n->out;
      k_conv_fwd<TA, true><<<g, CV_NT, 0, n->st>>>(a);
    } else {
      a.out = n->act[l];
      k_conv_fwd<TA, false><<<g, CV_NT, 0, n->st>>>(a);
    }
  }
  return net_check(n, "forward");
}

// split-K factor: enough CTAs for ~2 per SM, at most one K chunk each
int tc_ksplit(const NetLayer& L, int B) {
  const long long tiles = ((long long)B * L.hout * L.wout + 127) / 128;
  const int nchunk = (L.ci * 9 + TC_KC - 1) / TC_KC;
  long long ks = (2 * 148 + tiles - 1) / tiles;
  if (ks > nchunk) ks = nchunk;
  if (ks < 1) ks = 1;
  return (int)ks;
}

// largest split-K scratch over every batch size up to max_batch (a smaller
// batch can split K further)
size_t tc_part_size(int max_batch) {
  size_t m = 0;
  for (int B = 1; B <= max_batch; ++B)
    for (int l = 0; l < NET_LAYERS; ++l) {
      const NetLayer L = net_layer(l);
      const int ks = tc_ksplit(L, B);
      if (ks > 1) m = std::max(m, (size_t)ks * L.co * B * L.hout * L.wout);
    }
  return m;
}

template <int NP, bool NHWC = false>
void launch_conv_tc(ptycho_net* n, const ConvArgs& a, const NetLayer& L, bool out_f32) {
  const long long npix = (long long)a.B * a.hout * a.wout;
  const int ks = tc_ksplit(L, a.B);
  const dim3 g((unsigned)((npix + 127) / 128), (unsigned)ks);
  if (out_f32) k_conv_fwd_tc<true, NP, NHWC><<<g, 128, conv_tc_smem<NP>(), n->st>>>(a, ks, n->tc_part, n->err_flag);
  else k_conv_fwd_tc<false, NP, NHWC><<<g, 128, conv_tc_smem<NP>(), n->st>>>(a, ks, n->tc_part, n->err_flag);
  if (ks > 1) {
    const long long tot = npix * a.co;
    const unsigned rb = (unsigned)std::min<long long>((tot + 255) / 256, 4 * 1184);
    if (out_f32) k_conv_tc_reduce<true, NHWC><<<rb, 256, 0, n->st>>>(a, ks, n->tc_part);
    else k_conv_tc_reduce<false, NHWC><<<rb, 256, 0, n->st>>>(a, ks, n->tc_part);
  }
}

// Backward on the tensor cores (net_bwd_tc.cuh).  Pixel splits of the
// weight gradient: about as many CTAs as fit on the SMs at once (two per SM
// for the 144-wide tile, six for the one-channel one), within the partial
// buffer.
int bw_tc_nt(const NetLayer& L) { return L.ci == 1 ? BW_NT1 : BW_NT; }
int bw_tc_tiles(const NetLayer& L) {
  const int nt = bw_tc_nt(L);
  return ((L.co + 127) / 128) * ((L.ci * 9 + nt - 1) / nt);
}
long long bw_tc_want(const NetLayer& L) { return (bw_tc_nt(L) == BW_NT ? 2 : 6) * 148LL; }
int bw_tc_splits(const NetLayer& L, int B, size_t wpart_n) {
  const int tiles = bw_tc_tiles(L);
  const long long nchunk = ((long long)B * L.hout * L.wout + BW_KC - 1) / BW_KC;
  long long s = (bw_tc_want(L) + tiles - 1) / tiles;
  s = std::min<long long>(s, nchunk);
  s = std::min<long long>(s, (long long)(wpart_n / ((size_t)L.co * L.ci * 9)));
  return (int)std::max<long long>(s, 1);
}

// The parity-class data gradient of the stride-2 layers takes even input
// sizes, outputs of half the size and co a multiple of 8.
constexpr bool s2_layers_ok(int l = 0) {
  return l == NET_LAYERS ? true
                         : ((net_layer(l).stride != 2 ||
                             (net_layer(l).hin % 2 == 0 && net_layer(l).win % 2 == 0 &&
                              net_layer(l).hout == net_layer(l).hin / 2 && net_layer(l).wout == net_layer(l).win / 2 &&
                              net_layer(l).co % 8 == 0 && !net_layer(l).up)) &&
                            s2_layers_ok(l + 1));
}
static_assert(s2_layers_ok(), "stride-2 layer shapes");
// The tap-major gathers take a channel as k & (ci - 1) from 8 channels on.
constexpr bool ci_pow2(int l = 0) {
  return l == NET_LAYERS ? true
                         : ((net_layer(l).ci < 8 || (net_layer(l).ci & (net_layer(l).ci - 1)) == 0) && ci_pow2(l + 1));
}
static_assert(ci_pow2(), "input channels a power of two");

// K splits of the data gradient over co * 9 (deep layers have few pixels).
// Stride 2: four parity classes of B hin win / 4 pixels each, at most four
// taps per class.
int bd_tc_splits(const NetLayer& L, int B) {
  const bool s2 = L.stride == 2;
  const long long tiles = s2 ? 4 * (((long long)B * (L.hin / 2) * (L.win / 2) + 127) / 128)
                             : ((long long)B * L.hin * L.win + 127) / 128;
  const int nchunk = (L.co * (s2 ? 4 : 9) + BD_KC - 1) / BD_KC;
  long long ks = (2 * 148 + tiles - 1) / tiles;
  if (ks > nchunk) ks = nchunk;
  if (ks < 1) ks = 1;
  return (int)ks;
}

size_t bd_part_size(int max_batch) {
  size_t m = 0;
  for (int B = 1; B <= max_batch; ++B)
    for (int l = 1; l < NET_LAYERS; ++l) {
      const NetLayer L = net_layer(l);
      const int ks = bd_tc_splits(L, B);
      if (ks > 1) m = std::max(m, (size_t)ks * L.ci * B * L.hin * L.win);
    }
  return m;
}

template <int NP>
void launch_bwd_data_tc(ptycho_net* n, const ConvArgs& a, const NetLayer& L) {
  const long long npix = (long long)a.B * a.hin * a.win;
  const int ks = bd_tc_splits(L, a.B);
  if (L.stride == 2) {  // by parity class (even sizes, co a multiple of 8: the layer table)
    const long long tiles = ((long long)a.B * (L.hin / 2) * (L.win / 2) + 127) / 128;
    const dim3 g((unsigned)(4 * tiles), (unsigned)ks);
    k_conv_bwd_data_s2_tc<__nv_bfloat16, NP><<<g, 128, bd_s2_tc_smem<__nv_bfloat16, NP>(), n->st>>>(
        a, ks, n->bd_part, n->err_flag);
  } else {
    const dim3 g((unsigned)((npix + 127) / 128), (unsigned)ks);
    k_conv_bwd_data_tc<__nv_bfloat16, NP><<<g, 128, bd_tc_smem<NP>(), n->st>>>(a, ks, n->bd_part, n->err_flag);
  }
  if (ks > 1) {
    const unsigned rb = (unsigned)std::min<long long>((npix * a.ci + 255) / 256, 4 * 1184);
    k_bwd_data_reduce<__nv_bfloat16><<<rb, 256, 0, n->st>>>(a, ks, n->bd_part);
  }
}

// Inference forward (predict, warm start): the tensor-core convolutions on
// channel-last activations with tap-major weights (see k_conv_fwd_tc).  The
// sums run in another order than the training forward, so the two agree to
// FP32 rounding, then BF16 rounding per layer.
static_assert(net_layer(0).ci == 1 && net_layer(0).co == 16 && net_layer(0).relu, "first-layer kernel shape");
static_assert(net_layer(NET_LAYERS - 1).ci == 16 && net_layer(NET_LAYERS - 1).co == 2 &&
                  !net_layer(NET_LAYERS - 1).relu && !net_layer(NET_LAYERS - 1).up,
              "last-layer kernel shape");

// The tap-major weight copy, rebuilt from wb after the weights were set from
// the host (AdamW keeps it current afterwards).
void net_refresh_wt(ptycho_net* n) {
  if (n->wt_valid) return;
  for (int l = 0; l < NET_LAYERS; ++l) {
    const NetLayer L = net_layer(l);
    k_perm_weights<<<256, 256, 0, n->st>>>(n->wb + n->wb_off[l], n->wt + n->wb_off[l], L.co, L.ci);
  }
  n->wt_valid = true;
}

int net_infer(ptycho_net* n, int B) {
  net_refresh_wt(n);
  for (int l = 0; l < NET_LAYERS; ++l) {
    const NetLayer L = net_layer(l);
    ConvArgs a = conv_args(n, l, B);
    a.w = n->wt + n->wb_off[l];
    const bool last = l == NET_LAYERS - 1;
    a.out = last ? (void*)n->out : n->act[l];
    if (l == 0 || last) {  // 1 -> 16 and 16 -> 2 channels: CUDA cores
      const int npix = B * L.hout * L.wout;
      const unsigned g = (unsigned)std::min(4 * 148 * 8, (npix + 255) / 256);
      if (l == 0) k_conv_first_nhwc<<<g, 256, 0, n->st>>>(a);
      else k_conv_last_nhwc<<<g, 256, 0, n->st>>>(a);
      continue;
    }
    const int np = L.co <= 16 ? 16 : L.co;
    switch (np) {
      case 16: launch_conv_tc<16, true>(n, a, L, last); break;
      case 32: launch_conv_tc<32, true>(n, a, L, last); break;
      case 64: launch_conv_tc<64, true>(n, a, L, last); break;
      case 128: launch_conv_tc<128, true>(n, a, L, last); break;
      default: launch_conv_tc<256, true>(n, a, L, last); break;
    }
  }
  return net_check(n, "inference forward (tensor cores)");
}

int net_forward_tc(ptycho_net* n, int B) {
  net_refresh_wt(n);
  for (int l = 0; l < NET_LAYERS; ++l) {
    const NetLayer L = net_layer(l);
    ConvArgs a = conv_args(n, l, B);
    const bool last = l == NET_LAYERS - 1;
    a.out = last ? (void*)n->out : n->act[l];
    if (l == 0) {
      // the 1 -> 16 layer (144 FMAs per pixel) on CUDA cores, as in
      // inference: its tensor-core K chunk is 9 / 64 full (47 against 85 us
      // per step; the 16 -> 2 layer measured the other way, 71 against 52 us)
      const dim3 g((unsigned)(((long long)B * L.hout * L.wout + CV_NT - 1) / CV_NT),
                   (unsigned)((L.co + CV_CO - 1) / CV_CO));
      k_conv_fwd<__nv_bfloat16, false><<<g, CV_NT, 0, n->st>>>(a);
      continue;
    }
    if (L.ci >= 8) a.w = n->wt + n->wb_off[l];  // the NCHW gather takes tap-major k from 8 channels on
    const int np = L.co <= 16 ? 16 : L.co;
    switch (np) {
      case 16: launch_conv_tc<16>(n, a, L, last); break;
      case 32: launch_conv_tc<32>(n, a, L, last); break;
      case 64: launch_conv_tc<64>(n, a, L, last); break;
      case 128: launch_conv_tc<128>(n, a, L, last); break;
      default: launch_conv_tc<256>(n, a, L, last); break;
    }
  }
  return net_check(n, "forward (tensor cores)");
}

int net_forward(ptycho_net* n, int B) {
  if (n->f32) return net_forward_t<float>(n, B);
  return n->tc ? net_forward_tc(n, B) : net_forward_t<__nv_bfloat16>(n, B);
}

// Forward pass for predictions only (no backward pass follows).
int net_predict_forward(ptycho_net* n, int B) { return n->tc ? net_infer(n, B) : net_forward(n, B); }

// Loss against targets and all parameter gradients (into n->grads).
int net_backward(ptycho_net* n, const float* targets, int B, double* loss) {
  const size_t nout = (size_t)B * 2 * NET_OUT * NET_OUT;
  const int lb = 256;
  k_net_loss<<<lb, CV_NT, 0, n->st>>>(n->out, targets, nout, 1.f / (float)nout, n->delta[0], n->lpart);
  int cur = 0;
  // Per layer the bias gradient (it reads only this layer's delta) runs on
  // the side stream beside the weight gradient, and the weight gradient's
  // split sums beside the data gradient; the next layer's weight gradient
  // (which reuses the split buffer) and data gradient (which overwrites this
  // delta) wait for both.
  for (int l = NET_LAYERS - 1; l >= 0; --l) {
    const NetLayer L = net_layer(l);
    ConvArgs a = conv_args(n, l, B);
    a.dout = n->delta[cur];
    a.wpart = n->wpart;
    const long long npo = (long long)B * L.hout * L.wout;
    int nchunk = (int)((npo + BW_CHUNK - 1) / BW_CHUNK);
    if (l < NET_LAYERS - 1) cudaStreamWaitEvent(n->st, n->ev_join, 0);
    cudaEventRecord(n->ev_fork1, n->st);
    cudaStreamWaitEvent(n->st_side, n->ev_fork1, 0);
    {  // bias gradient: about four CTAs per SM, slices of >= 4096 deltas
      const int tot = B * L.hout * L.wout;
      const int nsl = std::max(1, std::min({(4 * 148 + L.co - 1) / L.co, (tot + 4095) / 4096, NET_BPART / L.co}));
      k_bias_grad_part<<<dim3((unsigned)L.co, (unsigned)nsl), CV_NT, 0, n->st_side>>>(n->delta[cur], B, L.co,
                                                                                    L.hout * L.wout, nsl, n->bpart);
      k_bias_grad_sum<<<(L.co + 255) / 256, 256, 0, n->st_side>>>(n->bpart, nsl, L.co, n->grads + n->b_off[l]);
    }
    if (n->tc) {  // tensor cores: pixel splits of (co tile x k tile) GEMMs
      nchunk = bw_tc_splits(L, B, n->wpart_n);
      const dim3 g((unsigned)bw_tc_tiles(L), (unsigned)nchunk);
      if (bw_tc_nt(L) == BW_NT1)
        k_conv_bwd_w_tc<__nv_bfloat16, BW_NT1><<<g, 128, bw_tc_smem_launch<BW_NT1>(), n->st>>>(a, nchunk, n->err_flag);
      else
        k_conv_bwd_w_tc<__nv_bfloat16, BW_NT><<<g, 128, bw_tc_smem_launch<BW_NT>(), n->st>>>(a, nchunk, n->err_flag);
    } else {
      const int nciq = (L.ci + BW_CI - 1) / BW_CI;
      if (n->f32) k_conv_bwd_w<float><<<dim3((unsigned)(L.co * nciq), (unsigned)nchunk), CV_NT, 0, n->st>>>(a);
      else k_conv_bwd_w<__nv_bfloat16><<<dim3((unsigned)(L.co * nciq), (unsigned)nchunk), CV_NT, 0, n->st>>>(a);
    }
    const size_t nw = (size_t)L.co * L.ci * 9;
    cudaEventRecord(n->ev_fork2, n->st);
    cudaStreamWaitEvent(n->st_side, n->ev_fork2, 0);
    if (nchunk >= 32 && nw <= 65536)  // few weights, many chunks: a warp per weight
      k_sum_chunks_warp<<<(unsigned)((nw + 7) / 8), 256, 0, n->st_side>>>(n->wpart, nchunk, nw,
                                                                          n->grads + n->w_off[l]);
    else
      k_sum_chunks<<<(unsigned)std::min<size_t>((nw + 255) / 256, 1184), 256, 0, n->st_side>>>(
          n->wpart, nchunk, nw, n->grads + n->w_off[l]);
    cudaEventRecord(n->ev_join, n->st_side);
    if (l > 0) {
      a.din = n->delta[cur ^ 1];
      a.mask = net_layer(l - 1).relu ? n->act[l - 1] : nullptr;
      // the last layer's data gradient (2 output channels: K = 18 of a 64-wide
      // chunk) on CUDA cores: 28.6k against 28.3k frames/s; the first
      // stride-2 layer's measured the other way (24.6k)
      if (n->tc && l != NET_LAYERS - 1) {
        switch (L.ci <= 16 ? 16 : L.ci) {
          case 16: launch_bwd_data_tc<16>(n, a, L); break;
          case 32: launch_bwd_data_tc<32>(n, a, L); break;
          case 64: launch_bwd_data_tc<64>(n, a, L); break;
          case 128: launch_bwd_data_tc<128>(n, a, L); break;
          default: launch_bwd_data_tc<256>(n, a, L); break;
        }
      } else {
        const dim3 g((unsigned)(((long long)B * L.hin * L.win + CV_NT - 1) / CV_NT),
                     (unsigned)((L.ci + CV_CI - 1) / CV_CI));
        if (n->f32) k_conv_bwd_data<float><<<g, CV_NT, 0, n->st>>>(a);
        else k_conv_bwd_data<__nv_bfloat16><<<g, CV_NT, 0, n->st>>>(a);
      }
      cur ^= 1;
    }
  }
  cudaStreamWaitEvent(n->st, n->ev_join, 0);  // every gradient is in place
  if (int r = net_check(n, "backward")) return r;
  if (loss) {
    double part[lb];
    cudaError_t e = cudaMemcpyAsync(part, n->lpart, sizeof part, cudaMemcpyDeviceToHost, n->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(n->st);
    if (e != cudaSuccess) return nfail(n, PTYCHO_ERR_CUDA, "loss: %s", cudaGetErrorString(e));
    double s = 0.0;
    for (int i = 0; i < lb; ++i) s += part[i];
    *loss = s;
  }
  return 0;
}

int net_input_src(ptycho_net* n, const void* src, int src_fft, int istore, const float* scale, int j0, int B) {
  if (n->f32)
    k_net_input<float><<<1184, 256, 0, n->st>>>(src, src_fft, istore, scale, j0, B, NET_IN, (float*)n->x);
  else
    k_net_input<__nv_bfloat16><<<1184, 256, 0, n->st>>>(src, src_fft, istore, scale, j0, B, NET_IN,
                                                        (__nv_bfloat16*)n->x);
  return net_check(n, "input");
}

int net_input(ptycho_net* n, const float* intensities, int B) {
  return net_input_src(n, intensities, 0, 0, nullptr, 0, B);
}

// SplitMix64-driven Box-Muller normals for the initial weights.
double net_normal(uint64_t& s) {
  auto next = [&]() {
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  const double u1 = ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  const double u2 = ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}

int net_upload_params(ptycho_net* n, const float* host) {
  std::vector<__nv_bfloat16> wb(n->n_w);
  for (int l = 0; l < NET_LAYERS; ++l) {
    const NetLayer L = net_layer(l);
    const long long nw = (long long)L.co * L.ci * 9;
    for (long long i = 0; i < nw; ++i) wb[n->wb_off[l] + i] = __float2bfloat16_rn(host[n->w_off[l] + i]);
  }
  cudaError_t e = cudaMemcpy(n->params, host, n->n_params * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(n->wb, wb.data(), n->n_w * sizeof(__nv_bfloat16), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return nfail(n, PTYCHO_ERR_CUDA, "parameter upload: %s", cudaGetErrorString(e));
  n->wt_valid = false;
  return 0;
}

}  // namespace

extern "C" {

int ptycho_net_create(ptycho_net** out, unsigned long long seed, int max_batch, int flags, void* stream) {
  if (!out || max_batch < 1 || max_batch > 4096 ||
      (flags & ~(PTYCHO_NET_F32_ACTIVATIONS | PTYCHO_NET_CUDA_CORES)))
    return nfail(nullptr, PTYCHO_ERR_ARG, "bad arguments");
  *out = nullptr;
  ptycho_net* n = new ptycho_net();
  n->f32 = (flags & PTYCHO_NET_F32_ACTIVATIONS) != 0;
  n->tc = !n->f32 && !(flags & PTYCHO_NET_CUDA_CORES);
  n->st = (cudaStream_t)stream;
  n->max_batch = max_batch;
  long long off = 0, woff = 0;
  for (int l = 0; l < NET_LAYERS; ++l) {
    const NetLayer L = net_layer(l);
    n->w_off[l] = off;
    off += (long long)L.co * L.ci * 9;
    n->b_off[l] = off;
    off += L.co;
    n->wb_off[l] = woff;
    woff += (long long)L.co * L.ci * 9;
  }
  n->n_params = off;
  n->n_w = woff;
  size_t maxd = 0, maxpart = 0;
  for (int l = 0; l < NET_LAYERS; ++l) {
    const NetLayer L = net_layer(l);
    maxd = std::max(maxd, (size_t)max_batch * L.co * L.hout * L.wout);
    maxd = std::max(maxd, (size_t)max_batch * L.ci * L.hin * L.win);
    const long long npo = (long long)max_batch * L.hout * L.wout;
    maxpart = std::max(maxpart, (size_t)((npo + BW_CHUNK - 1) / BW_CHUNK) * L.co * L.ci * 9);
    // the tensor-core weight gradient: about two CTAs per SM of pixel splits
    const long long tiles = bw_tc_tiles(L);
    const long long want = std::min<long long>((bw_tc_want(L) + tiles - 1) / tiles, (npo + BW_KC - 1) / BW_KC);
    maxpart = std::max(maxpart, (size_t)want * L.co * L.ci * 9);
  }
  int r = 0;
  if (cudaStreamCreateWithFlags(&n->st_side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&n->ev_fork1, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&n->ev_fork2, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&n->ev_join, cudaEventDisableTiming) != cudaSuccess)
    r = nfail(n, PTYCHO_ERR_CUDA, "side stream: %s", cudaGetErrorString(cudaGetLastError()));
  if (!r) r = nalloc(n, &n->params, n->n_params);
  if (!r) r = nalloc(n, &n->grads, n->n_params);
  if (!r) r = nalloc(n, &n->m, n->n_params);
  if (!r) r = nalloc(n, &n->v, n->n_params);
  if (!r) r = nalloc(n, &n->wb, n->n_w);
  if (!r && n->tc) r = nalloc(n, &n->wt, n->n_w);
  if (!r) r = nalloc(n, &n->is_w, n->n_params);
  if (!r) r = nalloc(n, &n->wb_index, n->n_params);
  if (!r) r = nalloc(n, &n->wt_index, n->n_params);
  const size_t asz = n->f32 ? 4 : 2;
  if (!r) r = nalloc(n, (unsigned char**)&n->x, (size_t)max_batch * NET_IN * NET_IN * asz);
  for (int l = 0; l + 1 < NET_LAYERS && !r; ++l) r = nalloc(n, (unsigned char**)&n->act[l], act_size(l, max_batch) * asz);
  if (!r) r = nalloc(n, &n->out, act_size(NET_LAYERS - 1, max_batch));
  if (!r) r = nalloc(n, &n->delta[0], maxd);
  if (!r) r = nalloc(n, &n->delta[1], maxd);
  n->wpart_n = maxpart;
  if (!r) r = nalloc(n, &n->wpart, maxpart);
  if (!r) r = nalloc(n, &n->lpart, 256);
  if (!r) r = nalloc(n, &n->bpart, NET_BPART);
  if (!r) r = nalloc(n, &n->err_flag, 1);
  if (!r && cudaMemset(n->err_flag, 0, sizeof(int)) != cudaSuccess) r = nfail(n, PTYCHO_ERR_CUDA, "memset");
  if (!r && n->tc) {
    n->tc_part_n = tc_part_size(max_batch);
    if (n->tc_part_n) r = nalloc(n, &n->tc_part, n->tc_part_n);
    n->bd_part_n = bd_part_size(max_batch);
    if (!r && n->bd_part_n) r = nalloc(n, &n->bd_part, n->bd_part_n);
    cudaError_t e2 = cudaSuccess;
    auto setsm = [&](const void* f, size_t b) {
      if (e2 == cudaSuccess) e2 = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b);
    };
    setsm((const void*)k_conv_fwd_tc<false, 16>, conv_tc_smem<16>());
    setsm((const void*)k_conv_fwd_tc<true, 16>, conv_tc_smem<16>());
    setsm((const void*)k_conv_fwd_tc<false, 32>, conv_tc_smem<32>());
    setsm((const void*)k_conv_fwd_tc<true, 32>, conv_tc_smem<32>());
    setsm((const void*)k_conv_fwd_tc<false, 64>, conv_tc_smem<64>());
    setsm((const void*)k_conv_fwd_tc<true, 64>, conv_tc_smem<64>());
    setsm((const void*)k_conv_fwd_tc<false, 128>, conv_tc_smem<128>());
    setsm((const void*)k_conv_fwd_tc<true, 128>, conv_tc_smem<128>());
    setsm((const void*)k_conv_fwd_tc<false, 256>, conv_tc_smem<256>());
    setsm((const void*)k_conv_fwd_tc<true, 256>, conv_tc_smem<256>());
    setsm((const void*)k_conv_fwd_tc<false, 16, true>, conv_tc_smem<16>());
    setsm((const void*)k_conv_fwd_tc<true, 16, true>, conv_tc_smem<16>());
    setsm((const void*)k_conv_fwd_tc<false, 32, true>, conv_tc_smem<32>());
    setsm((const void*)k_conv_fwd_tc<true, 32, true>, conv_tc_smem<32>());
    setsm((const void*)k_conv_fwd_tc<false, 64, true>, conv_tc_smem<64>());
    setsm((const void*)k_conv_fwd_tc<true, 64, true>, conv_tc_smem<64>());
    setsm((const void*)k_conv_fwd_tc<false, 128, true>, conv_tc_smem<128>());
    setsm((const void*)k_conv_fwd_tc<true, 128, true>, conv_tc_smem<128>());
    setsm((const void*)k_conv_fwd_tc<false, 256, true>, conv_tc_smem<256>());
    setsm((const void*)k_conv_fwd_tc<true, 256, true>, conv_tc_smem<256>());
    setsm((const void*)k_conv_bwd_w_tc<__nv_bfloat16, BW_NT>, bw_tc_smem_launch<BW_NT>());
    setsm((const void*)k_conv_bwd_w_tc<__nv_bfloat16, BW_NT1>, bw_tc_smem_launch<BW_NT1>());
    setsm((const void*)k_conv_bwd_data_tc<__nv_bfloat16, 16>, bd_tc_smem<16>());
    setsm((const void*)k_conv_bwd_data_tc<__nv_bfloat16, 32>, bd_tc_smem<32>());
    setsm((const void*)k_conv_bwd_data_tc<__nv_bfloat16, 64>, bd_tc_smem<64>());
    setsm((const void*)k_conv_bwd_data_tc<__nv_bfloat16, 128>, bd_tc_smem<128>());
    setsm((const void*)k_conv_bwd_data_tc<__nv_bfloat16, 256>, bd_tc_smem<256>());
    setsm((const void*)k_conv_bwd_data_s2_tc<__nv_bfloat16, 16>, bd_s2_tc_smem<__nv_bfloat16, 16>());
    setsm((const void*)k_conv_bwd_data_s2_tc<__nv_bfloat16, 32>, bd_s2_tc_smem<__nv_bfloat16, 32>());
    setsm((const void*)k_conv_bwd_data_s2_tc<__nv_bfloat16, 64>, bd_s2_tc_smem<__nv_bfloat16, 64>());
    setsm((const void*)k_conv_bwd_data_s2_tc<__nv_bfloat16, 128>, bd_s2_tc_smem<__nv_bfloat16, 128>());
    setsm((const void*)k_conv_bwd_data_s2_tc<__nv_bfloat16, 256>, bd_s2_tc_smem<__nv_bfloat16, 256>());
    if (!r && e2 != cudaSuccess) r = nfail(n, PTYCHO_ERR_CUDA, "tensor-core kernel setup: %s", cudaGetErrorString(e2));
  }
  if (r) {
    g_net_error = n->err;
    ptycho_net_destroy(n);
    return r;
  }
  // He-normal weights (std = sqrt(2 / (9 ci))), zero biases, from SplitMix64(seed)
  std::vector<float> p(n->n_params, 0.f);
  std::vector<unsigned char> isw(n->n_params, 0);
  std::vector<int> idx(n->n_params, 0), tidx(n->n_params, 0);
  uint64_t s = seed;
  for (int l = 0; l < NET_LAYERS; ++l) {
    const NetLayer L = net_layer(l);
    const double sd = std::sqrt(2.0 / (9.0 * L.ci));
    const long long nw = (long long)L.co * L.ci * 9;
    for (long long i = 0; i < nw; ++i) {
      p[n->w_off[l] + i] = (float)(sd * net_normal(s));
      isw[n->w_off[l] + i] = 1;
      idx[n->w_off[l] + i] = (int)(n->wb_off[l] + i);
      // i = (o ci + c) 9 + t  ->  tap-major o 9 ci + t ci + c
      const long long o = i / (9LL * L.ci), c = (i / 9) % L.ci, t = i % 9;
      tidx[n->w_off[l] + i] = (int)(n->wb_off[l] + (o * 9 + t) * L.ci + c);
    }
  }
  cudaError_t e = cudaMemcpy(n->is_w, isw.data(), isw.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(n->wb_index, idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(n->wt_index, tidx.data(), tidx.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(n->m, 0, n->n_params * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(n->v, 0, n->n_params * sizeof(float));
  int rc = e == cudaSuccess ? net_upload_params(n, p.data()) : PTYCHO_ERR_CUDA;
  if (rc) {
    g_net_error = n->err.empty() ? std::string(cudaGetErrorString(e)) : n->err;
    ptycho_net_destroy(n);
    return rc;
  }
  *out = n;
  return PTYCHO_OK;
}

long long ptycho_net_num_params(const ptycho_net* n) { return n ? n->n_params : -1; }

int ptycho_net_get_params(ptycho_net* n, float* out) {
  if (!n || !out) return PTYCHO_ERR_ARG;
  cudaError_t e = cudaMemcpyAsync(out, n->params, n->n_params * sizeof(float), cudaMemcpyDeviceToHost, n->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(n->st);
  if (e != cudaSuccess) return nfail(n, PTYCHO_ERR_CUDA, "get_params: %s", cudaGetErrorString(e));
  return PTYCHO_OK;
}

int ptycho_net_set_params(ptycho_net* n, const float* in) {
  if (!n || !in) return PTYCHO_ERR_ARG;
  for (long long i = 0; i < n->n_params; ++i)
    if (!std::isfinite(in[i])) return nfail(n, PTYCHO_ERR_NONFINITE, "parameter %lld is not finite", i);
  if (cudaStreamSynchronize(n->st) != cudaSuccess) return nfail(n, PTYCHO_ERR_CUDA, "sync");
  n->adam_t = 0;
  cudaMemset(n->m, 0, n->n_params * sizeof(float));
  cudaMemset(n->v, 0, n->n_params * sizeof(float));
  return net_upload_params(n, in);
}

int ptycho_net_predict(ptycho_net* n, const float* intensities, int B, float* out) {
  if (!n || !intensities || !out) return PTYCHO_ERR_ARG;
  if (B < 1 || B > n->max_batch) return nfail(n, PTYCHO_ERR_ARG, "batch %d outside [1, %d]", B, n->max_batch);
  if (int r = net_input(n, intensities, B)) return r;
  if (int r = net_predict_forward(n, B)) return r;
  cudaError_t e = cudaMemcpyAsync(out, n->out, act_size(NET_LAYERS - 1, B) * sizeof(float), cudaMemcpyDeviceToDevice,
                                  n->st);
  if (e != cudaSuccess) return nfail(n, PTYCHO_ERR_CUDA, "predict: %s", cudaGetErrorString(e));
  return PTYCHO_OK;
}

int ptycho_net_gradients(ptycho_net* n, const float* intensities, const float* targets, int B, float* grads,
                         double* loss) {
  if (!n || !intensities || !targets) return PTYCHO_ERR_ARG;
  if (B < 1 || B > n->max_batch) return nfail(n, PTYCHO_ERR_ARG, "batch %d outside [1, %d]", B, n->max_batch);
  if (int r = net_input(n, intensities, B)) return r;
  if (int r = net_forward(n, B)) return r;
  if (int r = net_backward(n, targets, B, loss)) return r;
  if (grads) {
    cudaError_t e = cudaMemcpyAsync(grads, n->grads, n->n_params * sizeof(float), cudaMemcpyDeviceToHost, n->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(n->st);
    if (e != cudaSuccess) return nfail(n, PTYCHO_ERR_CUDA, "gradients: %s", cudaGetErrorString(e));
  }
  return PTYCHO_OK;
}

int ptycho_net_train_step(ptycho_net* n, const float* intensities, const float* targets, int B, float lr,
                          double* loss) {
  if (!n || !intensities || !targets) return PTYCHO_ERR_ARG;
  if (B < 1 || B > n->max_batch) return nfail(n, PTYCHO_ERR_ARG, "batch %d outside [1, %d]", B, n->max_batch);
  if (!(lr > 0.f) || !std::isfinite(lr)) return nfail(n, PTYCHO_ERR_ARG, "learning rate %g", lr);
  if (int r = net_input(n, intensities, B)) return r;
  if (int r = net_forward(n, B)) return r;
  if (int r = net_backward(n, targets, B, loss)) return r;
  n->adam_t++;
  AdamArgs a{};
  a.p = n->params;
  a.g = n->grads;
  a.m = n->m;
  a.v = n->v;
  a.wb = n->wb;
  a.is_w = n->is_w;
  a.wb_index = n->wb_index;
  // the tap-major copy follows each step once it is valid (every weight is
  // updated), so the training forward needs no separate permutation
  a.wt = n->wt_valid ? n->wt : nullptr;
  a.wt_index = n->wt_index;
  a.n = (size_t)n->n_params;
  a.lr = lr;
  a.b1 = 0.9f;
  a.b2 = 0.999f;
  a.eps = 1e-8f;
  a.wd = 1e-4f;
  a.c1 = (float)(1.0 - std::pow(0.9, (double)n->adam_t));
  a.c2 = (float)(1.0 - std::pow(0.999, (double)n->adam_t));
  k_adam<<<1184, 256, 0, n->st>>>(a);
  return net_check(n, "adam");
}

const char* ptycho_net_last_error(const ptycho_net* n) { return n ? n->err.c_str() : g_net_error.c_str(); }

void ptycho_net_destroy(ptycho_net* n) {
  if (!n) return;
  if (n->st) cudaStreamSynchronize(n->st);
  else cudaDeviceSynchronize();
  if (n->st_side) {
    cudaStreamSynchronize(n->st_side);
    cudaStreamDestroy(n->st_side);
  }
  for (cudaEvent_t e : {n->ev_fork1, n->ev_fork2, n->ev_join})
    if (e) cudaEventDestroy(e);
  void* bufs[] = {n->tc_part, n->bd_part, n->bpart, n->err_flag, n->params, n->grads, n->m,   n->v,        n->wb,       n->wt,       n->is_w,     n->wb_index, n->wt_index,
                  n->x,      n->out,   n->wpart, n->lpart, n->delta[0], n->delta[1]};
  for (void* b : bufs)
    if (b) cudaFree(b);
  for (int l = 0; l < NET_LAYERS; ++l)
    if (n->act[l]) cudaFree(n->act[l]);
  delete n;
}

int ptycho_object_patches(ptycho_ctx* ctx, float* out) {
  if (!ctx || !out) return PTYCHO_ERR_ARG;
  if (!ctx->have_pos) return fail(ctx, PTYCHO_ERR_STATE, "object_patches before set_positions");
  if (ctx->p.M < NET_OUT) return fail(ctx, PTYCHO_ERR_ARG, "M=%d is smaller than the %d-pixel patch", ctx->p.M, NET_OUT);
  return launch(ctx, "patch_targets", 0.0, [&] {
    k_patch_targets<<<1184, 256, 0, ctx->st>>>(ctx->O, ctx->p.obj_nx, ctx->pos, ctx->p.J, ctx->p.M, out);
  });
}

int ptycho_warm_start(ptycho_ctx* ctx, ptycho_net* n) {
  if (!ctx || !n) return PTYCHO_ERR_ARG;
  if (!ctx->have_data) return fail(ctx, PTYCHO_ERR_STATE, "warm_start before set_data");
  if (ctx->p.M != NET_IN) return fail(ctx, PTYCHO_ERR_UNSUPPORTED, "the network takes %d-pixel frames", NET_IN);
  // predictions for all positions, batch by batch (ordered on the context stream)
  const int J = ctx->p.J;
  float* pred = nullptr;
  if (int r = dalloc(ctx, &pred, (size_t)J * 2 * NET_OUT * NET_OUT)) return r;
  cudaEvent_t ev;
  cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  cudaEventRecord(ev, ctx->st);
  cudaStreamWaitEvent(n->st, ev, 0);
  int rc = 0;
  for (int j0 = 0; j0 < J && !rc; j0 += n->max_batch) {
    const int B = std::min(n->max_batch, J - j0);
    rc = net_input_src(n, ctx->amp, 1, ctx->p.istore, ctx->amp_scale, j0, B);
    if (!rc) rc = net_predict_forward(n, B);
    if (!rc && cudaMemcpyAsync(pred + (size_t)j0 * 2 * NET_OUT * NET_OUT, n->out,
                               act_size(NET_LAYERS - 1, B) * sizeof(float), cudaMemcpyDeviceToDevice,
                               n->st) != cudaSuccess)
      rc = PTYCHO_ERR_CUDA;
  }
  cudaEventRecord(ev, n->st);
  cudaStreamWaitEvent(ctx->st, ev, 0);
  cudaEventDestroy(ev);
  if (rc) {
    cudaFree(pred);
    return fail(ctx, rc, "warm start prediction: %s", n->err.c_str());
  }
  rc = launch(ctx, "stitch", 0.0, [&] {
    k_stitch<<<ctx->n_tiles, 256, 0, ctx->st>>>(ctx->O, ctx->p.obj_ny, ctx->p.obj_nx, ctx->ntx, ctx->tile_ptr,
                                               ctx->tile_list, ctx->pos, ctx->p.M, pred, TILE_Y, TILE_X);
  });
  cudaError_t e = cudaStreamSynchronize(ctx->st);
  cudaFree(pred);
  if (rc) return rc;
  if (e != cudaSuccess) return fail(ctx, PTYCHO_ERR_CUDA, "warm start: %s", cudaGetErrorString(e));
  ctx->psi_valid = false;
  return PTYCHO_OK;
}

}  // extern "C"
