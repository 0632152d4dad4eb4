// libmgq reunitarisation pass: every link of a field projected back onto SU(3)
// by Gram-Schmidt (rows 0 and 1 normalised and orthogonalised, row 2 =
// conj(row0 x row1)), the projection that the update kernels apply after every
// link update.  For FP32 fields the projection can run in FP32 or in FP64 (the
// result stored in FP32 either way): the pass measures what an FP64 projection
// costs and buys on this part.
#include "mgq_internal.h"
#include "mgq_stencil.cuh"

namespace mgq {

template <class T, int NP, bool F64>
__global__ void __launch_bounds__(128) k_reunitarize(Links<T, NP> U, Geom g) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 8 * g.Vh) return;
    const int mp = idx / g.Vh, h = idx - mp * g.Vh, mu = mp >> 1, par = mp & 1;
    M3<T> u = U.load(mu, par, h);
    if constexpr (F64 && sizeof(T) == 4) {
        M3<double> d;
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) d.e[i][j] = mk((double)u.e[i][j].re, (double)u.e[i][j].im);
        reunitarize(d);
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) u.e[i][j] = mk((T)d.e[i][j].re, (T)d.e[i][j].im);
    } else {
        reunitarize(u);
    }
    U.store(mu, par, h, u);
}

}  // namespace mgq

using namespace mgq;

extern "C" {

mgq_status mgq_reunitarize(mgq_lattice* lat, int fp64_projection, void* stream) {
    Trace trace("mgq_reunitarize");
    mgq_status s = check_lattice(lat, false, "mgq_reunitarize");
    if (s) return s;
    if (fp64_projection < 0 || fp64_projection > 1) return fail(MGQ_EINVAL, "mgq_reunitarize: fp64_projection must be 0 or 1");
    const Geom g = make_geom(lat->dims);
    cudaStream_t st = as_stream(stream);
    const int nb = (int)((8L * g.Vh + 127) / 128);
    dispatch_prec(lat->prec, [&]<class T, int NP>() {
        if (fp64_projection)
            k_reunitarize<T, NP, true><<<nb, 128, 0, st>>>(links_of<T, NP>(lat), g);
        else
            k_reunitarize<T, NP, false><<<nb, 128, 0, st>>>(links_of<T, NP>(lat), g);
    });
    return cuda_check("mgq_reunitarize");
}

}  // extern "C"
