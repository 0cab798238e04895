"""Seeded synthetic clustering inputs (Gaussian mixtures).

The paper evaluates on 23 real data sets (Sec. 5: 2 to 5,000 attributes,
7,797 to 10,500,000 rows) that are not available here; these seeded mixtures
stand in for them with the same kind of structure (well separated and
overlapping clusters, anisotropic covariances, skewed cluster sizes and
uniform outliers).  This module only draws data: it holds none of the
clustering arithmetic, and both the CUDA path and the test oracle consume its
output.

Recipe (one numpy PCG64 stream per data set, seeded by ``seed``):

* means uniform in [-10, 10]^n;
* isotropic components: sigma = 1; anisotropic: covariance Q diag(lam) Q^T
  with Q Haar-distributed (QR of a Gaussian matrix, sign-fixed) and lam
  uniform in [0.1, 4];
* weights equal, Dirichlet(alpha=1), or Zipf (w_i proportional to i^-s);
  component sizes by largest-remainder rounding of m * w;
* rows are in random order (the component labels are shuffled);
* outliers (a fraction of the rows) are uniform over the bounding box of the
  inliers.
"""
import numpy as np

# The five workloads: id -> parameters.  Sample-size policies and budgets of
# each workload live with the benchmark / tests that use them.
WORKLOADS = {
    "gmm_10k_n2_k5": dict(m=10_000, n=2, components=5, cov="iso", weights="equal",
                          outliers=0.0),
    "gmm_1m_n16_k25": dict(m=1_000_000, n=16, components=25, cov="aniso",
                           weights="dirichlet", outliers=0.0),
    "gmm_4m_n32_k50o": dict(m=4_000_000, n=32, components=50, cov="iso",
                            weights="equal", outliers=0.01),
    "gmm_10m_n64_k100z": dict(m=10_000_000, n=64, components=100, cov="iso",
                              weights="zipf", outliers=0.0),
}


def _counts(m, w):
    w = np.asarray(w, dtype=np.float64)
    w = w / w.sum()
    raw = m * w
    base = np.floor(raw).astype(np.int64)
    rem = int(m - base.sum())
    order = np.argsort(-(raw - base), kind="stable")
    base[order[:rem]] += 1
    return base


def _haar(rng, n):
    z = rng.standard_normal((n, n))
    q, r = np.linalg.qr(z)
    return q * np.sign(np.diag(r))[None, :]


def gaussian_mixture(m, n, components, seed, cov="iso", weights="equal",
                     outliers=0.0, zipf_s=1.2, return_labels=False):
    """float32 (m, n) rows from a seeded Gaussian mixture (see module doc)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    means = rng.uniform(-10.0, 10.0, size=(components, n))
    if weights == "equal":
        w = np.ones(components)
    elif weights == "dirichlet":
        w = rng.dirichlet(np.ones(components))
    elif weights == "zipf":
        w = np.arange(1, components + 1, dtype=np.float64) ** (-zipf_s)
    else:
        raise ValueError(weights)
    n_out = int(round(outliers * m))
    counts = _counts(m - n_out, w)
    labels = np.concatenate([np.repeat(np.arange(components), counts),
                             np.full(n_out, components)]).astype(np.int32)
    rng.shuffle(labels)
    X = np.empty((m, n), dtype=np.float32)
    for c in range(components):
        rows = np.nonzero(labels == c)[0]
        z = rng.standard_normal((rows.size, n), dtype=np.float32)
        if cov == "aniso":
            lam = rng.uniform(0.1, 4.0, size=n)
            A = (_haar(rng, n) * np.sqrt(lam)[None, :]).astype(np.float32)
            z = z @ A.T
        X[rows] = (means[c].astype(np.float32)[None, :] + z).astype(np.float32)
    if n_out:
        inl = labels < components
        lo = X[inl].min(axis=0)
        hi = X[inl].max(axis=0)
        rows = np.nonzero(~inl)[0]
        X[rows] = rng.uniform(lo, hi, size=(rows.size, n)).astype(np.float32)
    if return_labels:
        return X, labels
    return X


def workload(name, seed=None, m=None):
    """Data of a named workload (optionally with fewer rows for quick tests)."""
    p = dict(WORKLOADS[name])
    if m is not None:
        p["m"] = int(m)
    if seed is None:
        seed = 1000 + list(WORKLOADS).index(name) + 1
    return gaussian_mixture(p["m"], p["n"], p["components"], seed, cov=p["cov"],
                            weights=p["weights"], outliers=p["outliers"])


def gaussian_mixture_device(m, n, components, seed, outliers=0.0, device="cuda"):
    """float32 (m, n) rows of an isotropic Gaussian mixture drawn on a CUDA
    device with torch (fast enough for the serving stream's large data sets):
    means uniform in [-10, 10]^n, sigma = 1, equal weights (component of a row
    uniform), a fraction `outliers` of rows uniform over the inliers' bounding
    box.  Seeded by a torch generator on the device, so its stream differs
    from the numpy recipe above; it draws data only."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    means = torch.rand((components, n), generator=g, device=device) * 20.0 - 10.0
    comp = torch.randint(0, components, (m,), generator=g, device=device)
    X = means[comp] + torch.randn((m, n), generator=g, device=device)
    n_out = int(round(outliers * m))
    if n_out:
        lo = X[n_out:].min(dim=0).values
        hi = X[n_out:].max(dim=0).values
        X[:n_out] = lo + (hi - lo) * torch.rand((n_out, n), generator=g, device=device)
        X = X[torch.randperm(m, generator=g, device=device)]
    return X.contiguous()
