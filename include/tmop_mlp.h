/*
 * tmop_mlp.h -- C ABI of the learned initial-iterate proposal for TMOP Newton.
 *
 * The paper has no learned component: its Newton method (Section 3.4) starts
 * from the given mesh. This extension proposes a better starting iterate for
 * 2D structured order-k meshes with a small MLP that maps the positions of a
 * 3x3-element patch to the displacement of the nodes the centre element
 * owns; plain Newton then runs from the proposal, and the caller judges it by
 * F and min det A (falling back to the unmodified mesh when it is worse or
 * inverted).
 *
 * Conventions: a 2D order-k grid of nx x ny elements has (k nx + 1) x
 * (k ny + 1) nodes, x fastest; element e = ex + nx ey; positions are DEVICE
 * FP64 SoA with component stride ldx (node i of component c at c*ldx + i, so
 * several meshes can share one allocation). The element size is h = 1/nx.
 * Element e OWNS its local nodes (i, j), 0 <= i, j < k (global node
 * (k ex + i, k ey + j)); every node off the right and top boundary is owned
 * by exactly one element.
 *
 * Patch features of centre element e: the (3k+1)^2 nodes (k(ex-1) + a,
 * k(ey-1) + b), a, b = 0..3k, as (p - c) / h - r_ab, where c is the mean of
 * the centre element's four vertices and r_ab the same node's position in a
 * uniform patch (Gauss-Lobatto nodes inside each element) relative to its
 * centre, so a uniform patch has zero features; stored node-major (b, then
 * a), x before y, as bfloat16, zero-padded to the row length. Nodes outside
 * the grid are point reflections through the boundary node of the same grid
 * line (p_ghost = 2 p_boundary - p_mirror), x direction first.
 *
 * Every call returns a tmop_status code (include/tmop.h) and is asynchronous
 * on the given stream (cudaStream_t as void*).
 */
#ifndef TMOP_MLP_H
#define TMOP_MLP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Features of elements first .. first+count-1: feat DEVICE bf16 (uint16_t
 * bit patterns) [count][ldf], ldf >= 2 (3k+1)^2, ldf a multiple of 8. */
int tmop_patch_features(int order, int nx, int ny, const double* x, int ldx, int first, int count, uint16_t* feat,
                        int ldf, void* stream);

/* Training targets: (x1 - x0) / h at the 2 k^2 owned dofs of each element,
 * ordered (j, i, component): T DEVICE float [count][ldt], ldt >= 2 k^2. */
int tmop_patch_targets(int order, int nx, int ny, const double* x0, const double* x1, int ldx, int first, int count,
                       float* T, int ldt, void* stream);

/* Proposal: x_out = x0 + scale h Y at every owned dof that is not fixed, x0
 * elsewhere (scale 1 is the network's prediction; smaller scales damp it).
 * Y DEVICE float [nx*ny][ldy] in the target layout (all elements, in
 * order); fixed DEVICE uint8 [2][ldx] or NULL. x_out may not alias x0. */
int tmop_patch_apply(int order, int nx, int ny, const double* x0, const uint8_t* fixed, int ldx, const float* Y,
                     int ldy, double scale, double* x_out, void* stream);

/* Coarse stage of the proposal (not in the paper). The curved-boundary
 * optimum differs from the mapped lattice by a displacement of the whole
 * domain's scale that a 3x3-element patch cannot see; the proposal
 * therefore first solves the TMOP problem of the element-vertex grid (an
 * order-1 context, Newton of Section 3.4) and interpolates its vertex
 * displacement to the fine nodes, and the network predicts only the local
 * residual from there.
 * tmop_lattice_vertices: xv DEVICE [2][ldv] (vertex (i, j) at j (nx+1) + i)
 * = the positions x DEVICE [2][ldx] (component stride ldx) of the lattice
 * nodes (k i, k j) of a 2D order-k grid. */
int tmop_lattice_vertices(int order, int nx, int ny, const double* x, int ldx, double* xv, int ldv, void* stream);

/* x_out = x_in + P (xv1 - xv0) at the dofs that are not fixed, x_in at the
 * fixed ones; P interpolates a vertex field bilinearly on each element at
 * its Gauss-Lobatto lattice nodes. xv0, xv1 DEVICE [2][ldv]; x_in, x_out
 * DEVICE [2][ldx] (may alias); fixed DEVICE uint8 [2][ldx] or NULL. */
int tmop_lattice_prolong_add(int order, int nx, int ny, const double* xv0, const double* xv1, int ldv,
                             const double* x_in, const uint8_t* fixed, int ldx, double* x_out, void* stream);

/* The network: n_in -> n_hidden -> n_hidden -> n_out, ReLU between layers,
 * bfloat16 weights and activations with FP32 accumulation on the
 * fifth-generation tensor cores (tcgen05.mma, accumulators in tensor
 * memory), FP32 master weights and Adam state. A GEMM whose bounded wait for
 * its tensor-core work gives up (not expected) raises the network's fault
 * flag and writes NaN into its output tile, so the loss and every later
 * output are NaN; tmop_mlp_forward, tmop_mlp_check and tmop_mlp_get report
 * the flag as TMOP_ERR_CUDA (and clear it).
 * n_hidden must be a multiple of 64; n_in <= 1024, n_out <= 64. Weights are
 * initialised He-normal from seed (the last layer scaled by 0.1), biases 0. */
typedef struct tmop_mlp tmop_mlp;
int tmop_mlp_create(int n_in, int n_hidden, int n_out, uint64_t seed, tmop_mlp** out);
void tmop_mlp_destroy(tmop_mlp* net);

/* Row length the feature matrix must have for this network (n_in padded). */
int tmop_mlp_input_ld(const tmop_mlp* net);

/* Y = net(X): X DEVICE bf16 [batch][input_ld], Y DEVICE float [batch][ldy]
 * (ldy >= n_out). batch a multiple of 64. Synchronises the stream to read the
 * fault flag (TMOP_ERR_CUDA if a GEMM gave up). */
int tmop_mlp_forward(tmop_mlp* net, const uint16_t* X, int batch, float* Y, int ldy, void* stream);

/* Reads (stream-ordered; synchronises the stream) and clears the fault flag:
 * TMOP_ERR_CUDA if some GEMM since the last check gave up its bounded wait,
 * else TMOP_OK. Training loops call it once per epoch: the asynchronous
 * tmop_mlp_gradients / tmop_mlp_adam do not synchronise. */
int tmop_mlp_check(tmop_mlp* net, void* stream);

/* Loss L = (1/batch) sum |Y - T|^2 and all parameter gradients (kept inside
 * the network; tmop_mlp_get(..., 1, ...) reads them). T DEVICE float
 * [batch][ldt]. loss DEVICE double scalar, or NULL. */
int tmop_mlp_gradients(tmop_mlp* net, const uint16_t* X, const float* T, int ldt, int batch, double* loss,
                       void* stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) after tmop_mlp_gradients.
 * The step count and its bias corrections live on the device, so a training
 * step (tmop_mlp_gradients + tmop_mlp_adam, no host synchronisation) can be
 * captured in a CUDA graph and replayed; lr is fixed at capture. */
int tmop_mlp_adam(tmop_mlp* net, float lr, void* stream);

/* Parameters (which = 0) or gradients (which = 1) as HOST float32 in the
 * flat unpadded order W1 [h][in], b1, W2 [h][h], b2, W3 [out][h], b3.
 * Synchronises the stream of the last call. */
size_t tmop_mlp_num_params(const tmop_mlp* net);
int tmop_mlp_get(tmop_mlp* net, int which, float* host, size_t n);
int tmop_mlp_set(tmop_mlp* net, const float* host, size_t n);

#ifdef __cplusplus
}
#endif
#endif /* TMOP_MLP_H */
