"""Plain CPU oracle for competitive-sample-size Big-means (arXiv 2403.18766).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or
run anything in this package.  The product path (the CUDA library and its
Python binding) never imports it and never falls back to it.

The oracle restates the paper step by step in plain numpy + Python:

* ``rng``      -- Philox4x64-10 counter-based generator (Salmon et al., SC'11)
                  and the unbiased bounded-integer draw both sides consume.
* ``kmeans``   -- Eq. (1) objective, nearest-centroid assignment, Lloyd
                  K-means, greedy K-means++ with candidate trials (Sec. 4.1,
                  Sec. 5 settings).
* ``bigmeans`` -- Algorithm 1 (Sec. 4.2-4.3): competing workers with random
                  sample sizes, the improving-size list L, s_opt, the common
                  recheck and the final full assignment.

It shares no code with the CUDA path; the two meet only through the seeded
input generators and through the published definition of Philox.
"""
