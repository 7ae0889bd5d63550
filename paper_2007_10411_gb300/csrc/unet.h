// Learned right preconditioner: a linear 3-level convolutional U-Net on the
// 2-D or 3-D grid (internal interface of libjfnk).
//
// Network (channels 16 / 32 / 64, 3x3 convolutions, zero padding, no biases,
// no activations, so the map is linear and fixed once trained):
//   x (nf fields, padded to 16 channels)
//   L0a 16->16, L0b 16->16 = s0 | avgpool 2x2
//   L1a 16->32, L1b 32->32 = s1 | avgpool 2x2
//   L2a 32->64, L2b 64->64       | nearest upsample x2, concat s1 (96)
//   L1c 96->32                   | nearest upsample x2, concat s0 (48)
//   L0c 48->16, L0d 1x1 16->16 (first nf channels are the output fields)
// 2-D: nf = 4 (u, w, theta, p) on nz x nx.  3-D: nf = 5 (u, v, w, theta, p) on
// nz x ny x nx; every 3x3 convolution acts on each horizontal (y, x) plane,
// pooling averages 2x2x2 blocks and upsampling repeats each point 2x2x2, so
// the vertical coupling comes from the coarser levels.
// Activations are bfloat16 in NHWC layout; convolutions are implicit GEMMs on
// the tensor cores (mma m16n8k16, bfloat16 inputs, float32 accumulation);
// weight gradients accumulate in float32; Adam keeps float32 master weights.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

namespace jfnk {

struct UNet;

// Supported grids: 2-D (ny = 1) with nx, nz multiples of 32; 3-D with nx a
// multiple of 32, ny of 64 and nz of 4.
bool unet_grid_ok(int dim, int nx, int ny, int nz);

// Weights: seeded random, last layer zero.  balance[nf] > 0: per-field factors
// B; the convolutions see B x and the map is N(x) = B^-1 net(B x), so that the
// loss weighs the fields as the Jacobian does.
UNet* unet_create(int dim, int nx, int ny, int nz, const double* balance, unsigned long long seed,
                  cudaError_t* err);
void unet_destroy(UNet* net);
size_t unet_num_weights(const UNet* net);
cudaError_t unet_get_weights(UNet* net, float* host, cudaStream_t s);
cudaError_t unet_set_weights(UNet* net, const float* host, cudaStream_t s);

// Weights, flat float32 order: layers L0a, L0b, L1a, L1b, L2a, L2b, L1c, L0c,
// L0d; within a layer [tap][cout][cin], tap = ky * k + kx for a k x k kernel
// whose tap (ky, kx) reads the input pixel at offset (ky - k/2, kx - k/2)
// (rows = z, columns = x).

// y = N(x) (accumulate = 0) or y += N(x) (accumulate = 1) for nf float32 field
// planes of nz x nx (2-D) or nz x ny x nx (3-D) points, x fastest; y must not
// overlap x.  When skip is
// non-NULL and *skip != 0 at kernel run time, every kernel returns at entry.
cudaError_t unet_apply(UNet* net, const float* x, float* y, int accumulate, const int* skip, cudaStream_t s);
// The one-time work an apply does before its launches (composing the first
// layers' weights after they changed), so that a capture of unet_apply holds
// only the network's fixed launch sequence.
cudaError_t unet_prepare(UNet* net, cudaStream_t s);
// Changes whenever weights, training steps or the engine change what an apply computes.
unsigned long long unet_version(const UNet* net);
int unet_launches_per_apply();

// Convolution engine: 0 tcgen05.mma with TMEM accumulators (default), 1 the
// mma.sync path.  Both compute the same layers (float32 accumulation).
cudaError_t unet_set_engine(UNet* net, int engine);
int unet_engine(const UNet* net);

// Synchronises s and reports cudaErrorLaunchTimeout when a tensor-core wait of
// an earlier convolution timed out (the flag stays set).
cudaError_t unet_check(UNet* net, cudaStream_t s);

// Loss L = 1/2 ||B (N(x) - t)||^2 / ||B x||^2 and dL/dW (float32, flat order of
// unet_get_weights) for one pair; grads may be NULL (loss only).
cudaError_t unet_loss_grad(UNet* net, const float* x, const float* t, double* loss, float* grads_host,
                           cudaStream_t s);

// Adam on the pairs (X[i], T[i]) (each nf field planes, device),
// epochs passes in a fixed order; loss_hist (host, epochs, may be NULL)
// receives the mean loss of every epoch.
cudaError_t unet_train(UNet* net, const float* X, const float* T, int npairs, int epochs, float lr,
                       double* loss_hist, cudaStream_t s);

}  // namespace jfnk
