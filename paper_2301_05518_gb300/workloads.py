"""The synthetic workloads the tests and the benchmark share (sizes, seeds, N, sigma).

The paper measures on HISQ gauge configurations with colour wall and point
sources (Sec. 3-4, Fig. 1) and n = 30-80 smearing steps (Sec. 3, Sec. 6); its
volumes and sigma values sat in figures that did not survive.  These seeded
synthetic workloads keep that structure.  sigma follows the reading
sigma / N = 0.2 where no value is given.
"""

# 8^3 x 16, near-unit links exp(i 0.3 H), one colour-0 point source at the
# origin on t = 0, N = 10 steps on that slice, FP64, single vector.
SMALL_POINT = dict(dims=(8, 8, 8, 16), links="near", eps=0.3, gauge_seed=1000,
                   N=10, sigma=2.0, timeslice=0)

# 32^3 x 64, near-unit links (0.3), 3 colour point sources + 3 Gaussian
# vectors, N = 40 on every slice, FP64 and FP32 storage, one vector per launch.
MEDIUM_MIXED = dict(dims=(32, 32, 32, 64), links="near", eps=0.3, gauge_seed=1001, vec_seed=2001,
                    N=40, sigma=8.0)

# 48^3 x 64, Haar links, Gaussian multi-RHS batches, N = 40.
LARGE_MRHS = dict(dims=(48, 48, 48, 64), links="haar", gauge_seed=1002, vec_seed=2002,
                  N=40, sigma=8.0, batches=(12, 24, 48, 96))

# 64^3 x 96 (V = 25,165,824), near-unit links (0.2), W built in FP64 and
# rounded to FP32, 24 corner-wall sources (3 colours x 8 corners, t = 0),
# N = 80 on every slice.  The headline workload.
HEADLINE = dict(dims=(64, 64, 64, 96), links="near", eps=0.2, gauge_seed=1003, N=80, sigma=16.0,
                nvec=24, name="64^3x96 24 corner-wall sources N=80")

# Serving stream: resident 16^3x32, 32^3x64, 48^3x96 Haar fields; jobs of
# 1-24 Gaussian vectors, N ~ U{10..80}, sigma/N ~ U[0.05, 0.3], FP32/FP16.
SERVING = dict(configs=((16, 16, 16, 32), (32, 32, 32, 64), (48, 48, 48, 96)), gauge_seed=1004,
               vec_seed=2004, arrival_seed=3000, nvec=(1, 24), N=(10, 80), sigma_per_N=(0.05, 0.3),
               hbm_cap=120 * 2 ** 30)

# Sink smearing in the many-source pattern of the baryon measurement (Sec. 6):
# 72 sources/sinks smeared with one two-link field, n = 30.  Stand-in: 48^3 x 64
# near-unit links (0.2), 72 dense Gaussian vectors on every slice (24 solved
# propagators x 3 colour columns), sigma / N = 0.2, FP32 storage, one
# multi-RHS batch.
SINK_SMEAR = dict(dims=(48, 48, 48, 64), links="near", eps=0.2, gauge_seed=1005, vec_seed=2005,
                  N=30, sigma=6.0, nvec=72, name="48^3x64 72 dense sink vectors N=30")
