/*
 * nslct.h -- C ABI of libnslct: the 2D nonseparable discrete linear canonical
 * transform (NsDLCT) computed as the CM-CC-CM-CC chain of Pei & Huang
 * ("Two-dimensional nonseparable discrete linear canonical transform based on
 * CM-CC-CM-CC decomposition"), on NVIDIA GB300 (sm_103a).
 *
 * Problem statement followed (Sec. 2, first paragraph): an Nx x Ny input
 * g[m,n] = g(m dx, n dy) sampled on a centred grid (m = i - floor(Nx/2) for
 * storage row i, n = j - floor(Ny/2) for storage column j) is mapped to an
 * Nx x Ny output G[p,q] ~ G(p du, q dv) with du = dx, dv = dy (Sec. 2.A),
 * where G is the 2D NsLCT of Eq. Intro08 with the 4x4 ABCD matrix of
 * Eq. Intro04.
 *
 * The transform is the chain of Eq. HA28 (Sec. 4.B.1), applied right to left:
 *     CC^H  ->  CM^{C2}  ->  CC^{B'}  ->  CM^{C1}
 * with B' = B - AH, D' = D - CH, C2 = B'^{-1}(A - I), C1 = (D' - I)B'^{-1}
 * (Eq. Bnonsym08), CM the chirp multiplication of Eq. BasicCM12 and
 * CC^B = F^{-1} CM^{-B} F the chirp convolution of Eq. BasicCC20.
 *
 * Data: every field is a dense row-major [Nx][Ny] array of interleaved complex
 * values -- complex64 (float re, float im) for NSLCT_PREC_FP32 plans and
 * complex128 (double re, double im) for NSLCT_PREC_FP64 plans -- in DEVICE
 * memory of the device that was current when the plan was made. Row index i
 * runs along x, column index j along y. Buffers are owned by the caller.
 *
 * Streams: nslct_stream_t is ABI-identical to cudaStream_t (pass one directly;
 * NULL means the legacy default stream). Transform calls are asynchronous on
 * that stream: they return after enqueueing the kernels.
 *
 * Errors: every entry point returns 0 (NSLCT_OK) or one of the NSLCT_E_*
 * codes below; nslct_strerror() gives a static message. A call that fails
 * enqueues nothing and leaves the output untouched.
 *
 * Thread safety: a plan may be used from several host threads at once for
 * transforms on different output buffers; creating and destroying plans is
 * not synchronised against use of the same plan.
 */
#ifndef NSLCT_H_
#define NSLCT_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nslct_plan_s* nslct_plan_t;   /* opaque, owned by the library */
typedef struct CUstream_st* nslct_stream_t;  /* same type as cudaStream_t */

/* ---- error codes ---------------------------------------------------------- */
#define NSLCT_OK                0
#define NSLCT_E_ARG             1  /* null pointer, N < 2, spacing <= 0, NaN input */
#define NSLCT_E_NOT_SYMPLECTIC  2  /* ABCD violates Eq. Intro12 and no projection was asked */
#define NSLCT_E_INFEASIBLE      3  /* no symmetric H with |det B'| >= 1e-3 (Eq. Bnonsym32) */
#define NSLCT_E_SIZE            4  /* Nx or Ny not of the form 2^a 3^b with 8 <= N <= 4096, a >= 1, b <= 1 */
#define NSLCT_E_CUDA            5  /* a CUDA runtime call failed */
#define NSLCT_E_NOMEM           6  /* device or host allocation failed */
#define NSLCT_E_TIMEOUT         7  /* a bounded device-side wait expired */
#define NSLCT_E_UNSUPPORTED     8  /* flag combination not available */

/* ---- plan flags ----------------------------------------------------------- */
/* Choice of H (the free symmetric matrix of Eq. Bnonsym04). */
#define NSLCT_H_HA          0x0u   /* high-accuracy criterion, Eq. HA24 (default) */
#define NSLCT_H_LC          0x1u   /* low-complexity closed form, Eqs. LC08/LC10; HA if invalid */
#define NSLCT_H_USER        0x2u   /* H given by the caller (nslct_plan_ex) */
#define NSLCT_H_LC_Y        0x3u   /* Eq. LC10's H = (0,0;0,h) when valid, else as NSLCT_H_LC */
#define NSLCT_H_MASK        0x3u
/* Replace a nearly symplectic ABCD (e.g. one printed to 4 decimals) by a
 * nearby exactly symplectic one before planning. */
#define NSLCT_PROJECT_SP4   0x10u
/* Always run the five-pass chain. Without it, FP32 plans whose H is
 * (0,0;0,h) (Eq. LC10, or H = 0) run in three passes: CC^H then convolves
 * along y only and shares one row pass with CM^{C2} (see nslct_plan_passes). */
#define NSLCT_FULL_CHAIN    0x20u
/* nslct_plan_padded: return only the centred Nx x Ny region of the padded output. */
#define NSLCT_CROP_OUTPUT   0x40u
/* The CC-CM-CC-CM decomposition (Eq. CCCMCCCM16) instead of Eq. HA28: the
 * chain CM^{Ca}, CC^{B1'}, CM^{Cb}, CC^{H1} with B1' = B - H1 D,
 * Ca = B1'^-1 (A - H1 C - I), Cb = (D - I) B1'^-1. It is computed exactly as
 * the inverse chain of the type-1 plan of M^-1 with H = -H1 (Eqs.
 * CCCMCCCM20-30), and H1 is chosen by the same criterion (HA, LC or given):
 * nslct_plan_params and nslct_derive then report the type-1 factors of M^-1
 * (H = -H1), nslct_plan_info the caller's M with this flag set. */
#define NSLCT_TYPE2         0x80u
/* Eq. Reversible08: type 2 when tr(B) < 0, type 1 otherwise (tr B = 0, left
 * open by the paper, counts as type 1); nslct_plan_info reports the choice
 * through NSLCT_TYPE2. Neither flag combines with zero padding, batches or
 * nslct_backward (NSLCT_E_UNSUPPORTED). */
#define NSLCT_TYPE_BY_TRACE 0x1000u
/* Arithmetic of the transform. */
#define NSLCT_PREC_FP32     0x000u /* complex64 data, FP32 FFT arithmetic (default) */
#define NSLCT_PREC_FP64     0x100u /* complex128 data, FP64 arithmetic throughout */
/* complex64 data; the 1D DFTs of 4096-point lines run as two DFT-64 stages
 * (four-step) on the fifth-generation tensor cores (tcgen05, FP32
 * accumulators in tensor memory), those of 256..2048-point lines as
 * radix-16 DFT-16 products on the warp-level tensor cores; operands are split
 * into FP16 halves (x = x_hi + x_lo, W = W_hi + W_lo;
 * x_lo W_hi + x_hi W_lo + x_hi W_hi, FP32 accumulation) after exact
 * power-of-two scaling. Twiddles, chirps and scales stay FP32. Backward and
 * uneven-batch (nslct_plan_batch) calls of such a plan run in FP32. */
#define NSLCT_PREC_SPLIT_F16 0x200u
#define NSLCT_PREC_MASK     0xF00u

/*
 * nslct_plan -- derive the chain's parameters for one ABCD matrix and field size.
 *
 *   out      receives the new plan (set to NULL on failure).
 *   abcd     16 doubles, row-major 4x4 (a11 a12 b11 b12 / a21 a22 b21 b22 /
 *            c11 c12 d11 d12 / c21 c22 d21 d22), the layout of Eq. Intro04.
 *            Must satisfy Eq. Intro12 to 1e-9 * max(1, max|M|^2) unless
 *            NSLCT_PROJECT_SP4 is set.
 *   Nx, Ny   field size (rows, columns); see NSLCT_E_SIZE for the sizes the GPU
 *            path supports.
 *   dx, dy   sampling intervals (> 0). The paper's condition for the DFT case
 *            is dx^2 = 2 pi / Nx, dy^2 = 2 pi / Ny (Sec. 2.B).
 *   flags    NSLCT_H_*, NSLCT_PROJECT_SP4, NSLCT_FULL_CHAIN, NSLCT_TYPE2 or
 *            NSLCT_TYPE_BY_TRACE, NSLCT_PREC_*.
 *
 * All derivation (symplectic check/projection, the H criterion of Eq. HA24 or
 * the closed form of Eqs. LC08/LC10, B', D', C1, C2, fixed-point chirp
 * coefficients) runs on the host in FP64. The plan allocates small device
 * tables (twiddles) on the current device; it needs no per-call workspace.
 */
int nslct_plan(nslct_plan_t* out, const double abcd[16], int Nx, int Ny,
               double dx, double dy, unsigned flags);

/*
 * nslct_plan_ex -- as nslct_plan; with NSLCT_H_USER, h_user (4 doubles,
 * row-major 2x2, symmetrised) is used as H and must make B - AH symmetric
 * (to 1e-9 relative) and invertible, else NSLCT_E_INFEASIBLE. h_user is
 * ignored for the other NSLCT_H_* choices and may be NULL.
 */
int nslct_plan_ex(nslct_plan_t* out, const double abcd[16], int Nx, int Ny,
                  double dx, double dy, unsigned flags, const double* h_user);

/*
 * nslct_derive -- the host-only part of planning, for inspection: validates
 * (or projects) `abcd`, chooses H by `flags` (NSLCT_H_*; h_user as in
 * nslct_plan_ex) and writes the projected ABCD (16 doubles), H, B' = B - AH,
 * C1 = (D' - I)B'^{-1}, C2 = B'^{-1}(A - I) (4 doubles each, row-major) and the
 * Eq. HA24 objective gamma(C1) gamma(B') gamma(C2) gamma(H) (Eq. HA16).
 * Output pointers may be NULL. Touches no GPU. Same error codes as nslct_plan.
 */
int nslct_derive(const double abcd[16], unsigned flags, const double* h_user, double abcd_used[16],
                 double H[4], double Bp[4], double C1[4], double C2[4], double* objective);

/*
 * nslct_plan_params -- copy out the plan's decomposition (Eq. Bnonsym08):
 * H, B' = B - AH, C1 = (D' - I)B'^{-1} (the CM applied last) and
 * C2 = B'^{-1}(A - I) (the CM applied second), each 4 doubles row-major.
 * Any output pointer may be NULL. `field` must be 0 for single plans.
 */
int nslct_plan_params(nslct_plan_t plan, int field, double H[4], double Bp[4],
                      double C1[4], double C2[4]);

/*
 * nslct_plan_info -- field size (the padded grid for padded plans), the plan's
 * flags (NSLCT_TYPE2 set when the type-2 chain is in use) and the projected
 * ABCD the plan uses (abcd may be NULL).
 */
int nslct_plan_info(nslct_plan_t plan, int* Nx, int* Ny, unsigned* flags, double abcd[16]);

/*
 * nslct_forward -- out = L in, the NsDLCT of Eq. HA28 (of Eq. CCCMCCCM16 for
 * type-2 plans).
 *   in, out  device buffers of Nx*Ny complex elements (see "Data" above),
 *            16-byte aligned; padded plans: the shapes of nslct_plan_shape.
 *            in == out (in-place) is allowed except for padded plans;
 *            otherwise they must not overlap. `out` doubles as the chain's
 *            intermediate storage, so no workspace is allocated (padded plans
 *            with a smaller output use their own).
 * nslct_plan_passes() kernel passes (5, or 3) are enqueued on `stream`.
 */
int nslct_forward(nslct_plan_t plan, const void* in, void* out, nslct_stream_t stream);

/*
 * nslct_inverse -- out = L^{-1} in, the chain of Eq. CCCMCCCM04 (= Eq.
 * CCCMCCCM30): the forward chain reversed with every chirp matrix negated, which
 * inverts it exactly in exact arithmetic (Sec. 4.D). Same buffer rules as
 * nslct_forward. Because L is unitary (Sec. 6.B), this is also L^H.
 */
int nslct_inverse(nslct_plan_t plan, const void* in, void* out, nslct_stream_t stream);

/*
 * nslct_plan_padded -- zero padding (Sec. 2.A; Sec. 5.A pads the input to
 * (N + dN) x (N + dN) against aliasing): the chain runs on the Nx_pad x Ny_pad
 * grid (supported lengths, Nx_pad >= Nx, Ny_pad >= Ny), with the caller's
 * Nx x Ny input (even sizes) at the centre: its row i is row
 * i + Nx_pad/2 - Nx/2 of the grid, likewise for columns, and zeros elsewhere.
 * The zeros are never stored: the first pass reads only the input's rows and
 * the rest of each line is zero in shared memory. nslct_forward then reads an
 * Nx x Ny array and writes the whole Nx_pad x Ny_pad output, or, with
 * NSLCT_CROP_OUTPUT, only its centred Nx x Ny region (the last pass stores
 * that region alone). nslct_inverse maps the output's shape back to the
 * input's: it zero-pads its input the same way and returns the centred
 * Nx x Ny region, so inverse(forward(x)) = x without cropping. dx, dy are the
 * sample spacings of the input (kept on the padded grid); the frequency
 * spacings become 2 pi / (N_pad dx). The plan owns an Nx_pad x Ny_pad work
 * field. In-place calls are rejected (NSLCT_E_ARG); nslct_backward and
 * batches do not take padded plans (NSLCT_E_UNSUPPORTED).
 */
int nslct_plan_padded(nslct_plan_t* out, const double abcd[16], int Nx, int Ny, int Nx_pad, int Ny_pad,
                      double dx, double dy, unsigned flags);

/* nslct_plan_shape -- the caller-side shapes: input rows x cols and output
 * rows x cols (both Nx x Ny for unpadded plans). Any pointer may be null. */
int nslct_plan_shape(nslct_plan_t plan, int* in_rows, int* in_cols, int* out_rows, int* out_cols);

/*
 * nslct_forward_many / nslct_inverse_many -- the transform (or its inverse) of
 * nbatch fields with the same plan: field b is read at in + b * in_stride and
 * written at out + b * out_stride (strides in complex elements, >= Nx*Ny
 * when nbatch > 1, each field 16-byte aligned; in == out needs equal
 * strides). For FP32 plans whose lines are 256..4096 points each pass is one
 * launch over the whole batch; other plans launch each pass once per field.
 * Padded plans: NSLCT_E_UNSUPPORTED. Otherwise as nslct_forward / nslct_inverse.
 */
int nslct_forward_many(nslct_plan_t plan, int nbatch, const void* in, long long in_stride, void* out,
                       long long out_stride, nslct_stream_t stream);
int nslct_inverse_many(nslct_plan_t plan, int nbatch, const void* in, long long in_stride, void* out,
                       long long out_stride, nslct_stream_t stream);

/*
 * nslct_forward_group -- out[k] = L_k in[k] for n independent transforms
 * (plans on one device; any sizes and flags), enqueued alternately on
 * `stream` and on a library-owned side stream that forks from and joins back
 * to `stream`: each transform's passes fill the last partial wave and the
 * start-up of the other stream's, and everything is complete in `stream`
 * order when the call's work there completes. Buffer rules as nslct_forward
 * for each k; the pairs must not overlap one another. Concurrent calls on one
 * device share the side stream (serialising their side halves). Capturable.
 * The side stream is made on the first call per device and kept for the
 * life of the process (it does not survive cudaDeviceReset).
 */
int nslct_forward_group(int n, const nslct_plan_t* plans, const void* const* in, void* const* out,
                        nslct_stream_t stream);

/*
 * nslct_forward_masked -- out = mask .* (L in): the forward transform followed
 * by a pointwise filter in the NsLCT domain (the H1, H3 of Eqs. Add04/Add08),
 * multiplied in the last pass before the store, so it costs one read of the
 * mask instead of a separate pass. mask: device array of the output's shape
 * and type (row-major, 16-byte aligned), not modified; it must not overlap
 * `out`. Same errors as nslct_forward, NSLCT_E_ARG for a null or misaligned mask.
 */
int nslct_forward_masked(nslct_plan_t plan, const void* in, const void* mask, void* out, nslct_stream_t stream);

/*
 * nslct_plan_passes -- kernel passes per transform of this plan: 5, or 3 for
 * FP32 plans with H = (0,0;0,h) (unless NSLCT_FULL_CHAIN): then
 *   forward: row [FFT_y, chi_{-H}, IFFT_y, CM^{C2}, FFT_y], column [FFT_x, chi_{-B'},
 *            IFFT_x], row [IFFT_y, CM^{C1}];
 * the same operators as the five-pass chain, since with chi_H independent of
 * k_x the x transforms of CC^H cancel.
 */
int nslct_plan_passes(nslct_plan_t plan);

/*
 * nslct_forward_pass -- enqueue ONE of the kernel passes that make up
 * nslct_forward, for profiling and per-pass testing; calling passes
 * 0 .. nslct_plan_passes() - 1 in order on the same buffers gives exactly
 * nslct_forward's result. For five-pass plans:
 *   pass 0: row FFT of `in` (row-major) into `out` (2x2-tiled layout)
 *   pass 1: column FFT, chirp CM^{-H} at the frequency spacing, column IFFT
 *   pass 2: row IFFT, -1/(Nx Ny), CM^{C2}, row FFT
 *   pass 3: column FFT, chirp CM^{-B'}, column IFFT
 *   pass 4: row IFFT, -1/(Nx Ny), CM^{C1}, back to row-major in `out`
 * Passes 1..4 read and write `out` only (`in` must still be non-NULL).
 */
int nslct_forward_pass(nslct_plan_t plan, int pass, const void* in, void* out, nslct_stream_t stream);

/*
 * nslct_backward -- vector-Jacobian product of y = L x (nslct_forward) for a
 * real loss l(y), with gradients for the chain's parameters.
 *   grad_out   dl/dRe y + j dl/dIm y (device, Nx*Ny elements of the plan's type)
 *   y          the forward output L x (device, read only)
 *   grad_in    receives dl/dRe x + j dl/dIm x = L^H grad_out (device). L is
 *              unitary (Sec. 6.B), so this is the inverse chain of Eq.
 *              CCCMCCCM04 applied to grad_out.
 *   grad_theta NULL or a DEVICE pointer to 10 doubles: dl/dtheta for the
 *              parametrisation M(theta) = (I,0;C,I)(L,0;0,L^-T)(I,B;0,I) of the
 *              plan's ABCD, theta = (c11,c12,c22, l11,l12,l21,l22, b11,b12,b22)
 *              (C, B symmetric, L = A), with H following theta as in
 *              nslct_plan_theta. NSLCT_E_UNSUPPORTED if the plan's A is singular.
 *   grad_chirp NULL or a DEVICE pointer to 12 doubles: dl/d(h11,h12,h22,
 *              b'11,b'12,b'22, c1_11,c1_12,c1_22, c2_11,c2_12,c2_22) with the
 *              decomposition of Eq. Bnonsym08 held fixed (off-diagonal entries
 *              counted once, as they enter the chirp phases).
 *   workspace  NULL, or a device buffer of Nx*Ny elements the call may
 *              overwrite. With NULL, the plan makes one on the first call
 *              (cudaMalloc) and keeps it until nslct_destroy.
 * The forward intermediates are recomputed by running y back through the
 * inverse chain next to grad_out, so nothing is stored by nslct_forward. On the
 * first call with gradients the plan also allocates a small buffer of per-CTA
 * partial sums. Calls on one plan that overlap on the GPU share those buffers
 * and race. All device pointers must be 16-byte aligned. Padded and type-2
 * plans are not supported (NSLCT_E_UNSUPPORTED).
 */
int nslct_backward(nslct_plan_t plan, const void* grad_out, const void* y, void* grad_in,
                   double* grad_theta, double* grad_chirp, void* workspace, nslct_stream_t stream);

/*
 * nslct_backward_many -- nslct_backward for nbatch fields of one plan whose
 * loss is the sum of per-field terms (a batch with shared ABCD parameters):
 * grad_out, y, grad_in (and workspace, if given) hold nbatch fields `stride`
 * elements apart (>= Nx*Ny when nbatch > 1, 16-byte aligned fields);
 * grad_in gets each field's L^H grad_out, and grad_theta / grad_chirp the
 * gradients summed over the batch. Each dual pass is one launch over the
 * batch. The plan's own workspace and partial-sum buffer grow to the batch.
 */
int nslct_backward_many(nslct_plan_t plan, int nbatch, long long stride, const void* grad_out, const void* y,
                        void* grad_in, double* grad_theta, double* grad_chirp, void* workspace,
                        nslct_stream_t stream);

/*
 * nslct_backward_pass -- enqueue ONE of the five dual passes of
 * nslct_backward_many (same arguments, pass 0..4), for profiling and per-pass
 * timing. Each pass reads the previous pass's outputs:
 *   pass 0: grad_out and y (row-major) -> grad_in and the value-path workspace
 *   passes 1..4: grad_in and the workspace -> themselves
 * In pass 4 grad_in returns to row-major. Calling passes 0..4 in order gives
 * nslct_backward_many's grad_in. The per-CTA parameter sums land in the plan's
 * partial-sum buffer but are never finalised: no gradient for theta or the
 * chirps comes out of these calls. NSLCT_E_ARG for a pass outside 0..4,
 * otherwise as nslct_backward_many.
 */
int nslct_backward_pass(nslct_plan_t plan, int pass, int nbatch, long long stride, const void* grad_out,
                        const void* y, void* grad_in, void* workspace, nslct_stream_t stream);

/*
 * nslct_plan_theta -- plan for M(theta) (see nslct_backward) with H = h0 moved
 * onto the feasible plane of M(theta) along its normal:
 *   h = h0 + r (rhs - r.h0) / (r.r),  r = (-a21, a11 - a22, a12), rhs = b12 - b21,
 * the smooth H rule the parameter gradients differentiate. With h0 NULL, H is
 * chosen by the Eq. HA24 criterion instead. The NSLCT_H_* and
 * NSLCT_PROJECT_SP4 bits of `flags` are ignored; NSLCT_E_ARG if L is singular.
 */
int nslct_plan_theta(nslct_plan_t* out, const double theta[10], const double h0[4], int Nx, int Ny,
                     double dx, double dy, unsigned flags);

/*
 * nslct_plan_theta_set -- move a plan made by nslct_plan_theta with an h0 to
 * new parameters theta (10 doubles, as there), with H(theta) from the same h0:
 * the plan then equals nslct_plan_theta(theta, h0) of the same size, spacings
 * and flags. The derivation of Eqs. Intro12 and Bnonsym08 (M, H, B', C1, C2,
 * the Q0.64 chirp coefficients and the theta Jacobian) runs in FP64 on the
 * host; nothing is allocated and no CUDA call is made, so it may be called
 * between the steps of an optimisation loop at no device cost.
 * Transforms already enqueued keep the parameters they were enqueued with
 * (the chirps are kernel arguments); enqueueing on the plan from another
 * thread during the call is not allowed. NSLCT_E_UNSUPPORTED for plans not
 * made that way (h0 NULL, padded, type 2); NSLCT_E_ARG if L is singular or
 * theta not finite; NSLCT_E_INFEASIBLE if B' is singular at theta. On error
 * the plan is unchanged.
 */
int nslct_plan_theta_set(nslct_plan_t plan, const double theta[10]);

/* nslct_plan_theta_get -- theta of the plan's ABCD (NSLCT_E_UNSUPPORTED if A is singular). */
int nslct_plan_theta_get(nslct_plan_t plan, double theta[10]);

/*
 * nslct_backward_noalloc -- nslct_backward for callers that cannot allocate
 * device memory: code recording a CUDA graph (where cudaMalloc is not allowed
 * inside the capture), code under a caching allocator that must own every
 * allocation, or code with a fixed memory budget. The paper has no counterpart;
 * this is an interface variant of nslct_backward.
 *   grad_out, grad_in, grad_theta, grad_chirp   as in nslct_backward.
 *   y_inout    the forward output y (device). It doubles as the value-path
 *              buffer, so on return it holds L^{-1} y, the reconstructed input.
 *              It must not overlap grad_in (NSLCT_E_ARG).
 * The call makes no allocation of any kind. Its per-CTA partial sums go to a
 * fixed device array inside the library (4 x 2049 x 3 doubles, about 196 KB,
 * enough for every supported size; larger would return NSLCT_E_SIZE), which
 * every GPU that loads the library holds until the process exits. The first
 * call on a device (and the first after the device's context was reset) looks
 * that array's device address up (cudaGetSymbolAddress with the plan's device
 * current); make that first call before any stream capture. Each call rewrites all the array entries it reads, so nothing has
 * to be cleared between calls; but every call shares the one array, so calls
 * that overlap on the GPU (other streams, other threads, other plans) race.
 */
int nslct_backward_noalloc(nslct_plan_t plan, const void* grad_out, void* y_inout, void* grad_in,
                           double* grad_theta, double* grad_chirp, nslct_stream_t stream);

/* ---- batches of fields with uneven sizes ------------------------------------ */
typedef struct nslct_batch_s* nslct_batch_t;  /* opaque, owned by the library */

/*
 * nslct_plan_batch -- plans for `nfields` fields, field f of size Nx[f] x Ny[f]
 * with spacings dx[f], dy[f] and its own ABCD matrix abcd[16 f .. 16 f + 15]
 * (layout as in nslct_plan). NSLCT_PREC_FP32 only. Line lengths must be one of
 * 64, 96, 128, 192, 256, 384, 512, 768, 1024, 1536, 2048, 4096 (else
 * NSLCT_E_SIZE). Each field gets its own plan (reachable by nslct_batch_plan);
 * the batch also prepares per-pass work lists of (field, panel) items, longest
 * lines first.
 */
int nslct_plan_batch(nslct_batch_t* out, int nfields, const double* abcd, const int* Nx, const int* Ny,
                     const double* dx, const double* dy, unsigned flags);

/* nslct_batch_size / nslct_batch_plan -- field count; the plan of field `field` (owned by the batch). */
int nslct_batch_size(nslct_batch_t batch);
int nslct_batch_plan(nslct_batch_t batch, int field, nslct_plan_t* plan);

/*
 * nslct_batch_bind -- attach the fields' device buffers: in[f], out[f] (host
 * arrays of nfields device pointers; row-major fields as for nslct_forward,
 * 16-byte aligned). Uploads the pass descriptors (synchronous) and drops any
 * captured graph.
 */
int nslct_batch_bind(nslct_batch_t batch, const void* const* in, void* const* out);

/*
 * nslct_batch_forward -- out[f] = L_f in[f] for every bound field: one counter
 * reset and five persistent launches, one per pass of the chain, each covering
 * all fields (items handed out through an atomic counter); or, after
 * nslct_batch_capture, one launch of the captured CUDA graph.
 */
int nslct_batch_forward(nslct_batch_t batch, nslct_stream_t stream);

/* nslct_batch_capture -- capture the bound batch's launches on `stream` (not the
 * legacy default stream) into a CUDA graph that nslct_batch_forward then launches. */
int nslct_batch_capture(nslct_batch_t batch, nslct_stream_t stream);

/*
 * nslct_batch_set_split -- fields whose shorter side is >= `split` run through
 * their own plan's fused passes (as nslct_forward), enqueued before the batched
 * launches; the others stay in the batched launches. The default (2^30)
 * batches every field. Drops a captured graph. nslct_batch_get_split returns it.
 */
int nslct_batch_set_split(nslct_batch_t batch, int split);
int nslct_batch_get_split(nslct_batch_t batch);
/* nslct_batch_threads -- the CTA size of the batched kernels: 128 (four CTAs
 * per SM, power-of-two lines as packed pairs; the default when every line is
 * at most 2048 points; in column passes, 3*2^a lines run packed in a second
 * 128-thread kernel at three CTAs per SM, on a stream forked from and joined
 * back to the caller's), 256 (two CTAs per SM) or 512 (any length). */
int nslct_batch_threads(nslct_batch_t batch);
/* nslct_batch_set_threads -- pin the batched kernels' CTA size (128, 256 or
 * 512, else NSLCT_E_ARG). NSLCT_E_SIZE if some field has a line that size does
 * not handle (256: lines up to 2048; 128: up to 2048, power-of-two lines
 * packed in pairs). Drops a captured graph; a later nslct_batch_tune may
 * change it again. */
int nslct_batch_set_threads(nslct_batch_t batch, int threads);

/*
 * nslct_batch_tune -- autotune the split and the batched kernels' CTA size on
 * the bound buffers: for every distinct shorter side (and "batch everything"),
 * and each CTA size that handles every line, run one warm-up forward and
 * `iters` timed forwards on `stream` (CUDA events), keep the fastest, and
 * return it in *chosen (nullable) with its time per forward in
 * *ms_per_forward (nullable). Synchronises `stream`. Overwrites the bound
 * outputs; bindings with in[f] == out[f] are rejected (NSLCT_E_ARG) because
 * the repeated runs would feed outputs back in. Drops a captured graph.
 */
int nslct_batch_tune(nslct_batch_t batch, nslct_stream_t stream, int iters, int* chosen, float* ms_per_forward);

/*
 * nslct_batch_forward_pass -- enqueue ONE of the five passes of
 * nslct_batch_forward (pass 0..4, as in nslct_forward_pass), for profiling and
 * per-pass timing. The batched fields get one persistent launch; fields that
 * run alone (see nslct_batch_set_split) get their own nslct_forward_pass, on
 * `stream`. Calling passes 0..4 in order gives nslct_batch_forward's outputs.
 * Does not use a captured graph. NSLCT_E_ARG if the batch is unbound or the
 * pass is outside 0..4.
 */
int nslct_batch_forward_pass(nslct_batch_t batch, int pass, nslct_stream_t stream);

/* nslct_batch_forward_each -- the same transforms as per-field nslct_forward calls (5 launches per field). */
int nslct_batch_forward_each(nslct_batch_t batch, nslct_stream_t stream);

/* nslct_batch_destroy -- free the batch, its plans and its graph. */
int nslct_batch_destroy(nslct_batch_t batch);

/*
 * nslct_status -- synchronise with the plan's device (blocking) and report
 * whether any of its kernels gave up a bounded device-side wait since the last
 * call: NSLCT_OK, or NSLCT_E_TIMEOUT (the status word is cleared). A kernel
 * that gives up leaves its output incomplete instead of hanging the GPU.
 */
int nslct_status(nslct_plan_t plan);

/*
 * nslct_selftest_timeout -- exercise the bounded waits: enqueue the first pass
 * of `plan`'s forward chain with every panel's barrier expecting 16 bytes more
 * than its copies bring and a 1 ms limit, so that each CTA's wait expires,
 * sets the plan's status word and returns (every copy it issued still lands;
 * nothing faults or hangs). `out` receives no result. Afterwards
 * nslct_status reports NSLCT_E_TIMEOUT once and the plan works normally.
 * FP32 plans whose rows are 256..4096 points; in != out, 16-byte aligned.
 */
int nslct_selftest_timeout(nslct_plan_t plan, const void* in, void* out, nslct_stream_t stream);

/* nslct_destroy -- free a plan and its device tables (NULL is allowed). */
int nslct_destroy(nslct_plan_t plan);

/* nslct_strerror -- static description of an NSLCT_* code. */
const char* nslct_strerror(int code);

/* nslct_version -- library version string. */
const char* nslct_version(void);

#ifdef __cplusplus
}
#endif

#endif /* NSLCT_H_ */
