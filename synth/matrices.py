"""Seeded test matrices with prescribed spectra (see package docstring)."""
import numpy as np

# The five workloads: sizes, ranks, spectra, noise and seeds.  Seeds: the matrix
# generator uses 0xA000 + index, the Omega stream 0x5EED + index.
CONFIGS = {
    "c1_f64_2000x1000": dict(index=1, m=2000, n=1000, k=50, p=10, q=1, dtype="float64",
                             spectrum="exp20", r=1000, noise=0.0),
    "c2_f32_50000x20000": dict(index=2, m=50000, n=20000, k=200, p=20, q=2, dtype="float32",
                               spectrum="inv", r=2000, noise=1e-4),
    "c3_bf16_100000x50000": dict(index=3, m=100000, n=50000, k=500, p=50, q=2, dtype="bfloat16",
                                 spectrum="exp100", r=2000, noise=1e-4),
    "c5_f32_8192x4096": dict(index=5, m=8192, n=4096, k=64, p=16, q=2, dtype="float32",
                             spectrum="sqrtgap64", r=4096, noise=0.0),
}

# The batched workload: 512 FP32 problems, m ~ U[256, 4096], n ~ U[128, 2048]
# with n <= m, k drawn from {8, 16, 32, 64}, p = 8, q = 1, sigma_j = exp(-j/k).
BATCH_CONFIGS = {
    "c4_f32_batched512": dict(index=4, batch=512, m_range=(256, 4096), n_range=(128, 2048),
                              ks=(8, 16, 32, 64), p=8, q=1, dtype="float32", spectrum="expk"),
}


def batch_sizes(name, batch=None):
    """(ms, ns, ks) of a batched workload, drawn with the workload's seed."""
    c = BATCH_CONFIGS[name]
    b = c["batch"] if batch is None else batch
    rng = np.random.default_rng(0xA000 + c["index"])
    ms = rng.integers(c["m_range"][0], c["m_range"][1] + 1, size=b)
    ns = rng.integers(c["n_range"][0], c["n_range"][1] + 1, size=b)
    ns = np.minimum(ns, ms)
    ks = rng.choice(np.asarray(c["ks"]), size=b)
    ns = np.maximum(ns, ks + c["p"])     # l = k + p <= n
    return [int(x) for x in ms], [int(x) for x in ns], [int(x) for x in ks]


def make_batch_torch(ms, ns, ks, seed, device="cuda", tail=6):
    """A_i = U_i diag(sigma) V_i^T with sigma_j = exp(-j/k_i), j <= min(n_i, tail k_i)
    (the spectrum is cut where it falls below e^-tail), U_i and V_i orthonormalised
    Gaussian matrices drawn and factored on ``device`` (torch QR).  float32 list."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))

    def qr_q(X):
        try:
            return torch.linalg.qr(X)[0]
        except RuntimeError:   # no device LAPACK in this process: factor on the host
            return torch.linalg.qr(X.cpu())[0].to(X.device)

    out = []
    for m, n, k in zip(ms, ns, ks):
        r = int(min(n, tail * k))
        sig = torch.exp(-torch.arange(1, r + 1, device=device, dtype=torch.float64) / k)
        U = qr_q(torch.randn(m, r, generator=g, device=device, dtype=torch.float64))
        V = qr_q(torch.randn(n, r, generator=g, device=device, dtype=torch.float64))
        out.append(((U * sig[None, :]) @ V.T).to(torch.float32).contiguous())
    return out


def config(name):
    c = dict(CONFIGS[name])
    c["a_seed"] = 0xA000 + c["index"]
    c["omega_seed"] = 0x5EED + c["index"]
    c["l"] = c["k"] + c["p"]
    return c


def spectrum(kind, r, k=None):
    """Prescribed singular values sigma_1..sigma_r (float64, descending)."""
    j = np.arange(1, r + 1, dtype=np.float64)
    if kind == "exp20":                      # sigma_j = exp(-j/20)
        return np.exp(-j / 20.0)
    if kind == "inv":                        # sigma_j = 1/j
        return 1.0 / j
    if kind == "exp100":                     # sigma_j = exp(-j/100) + 1e-3
        return np.exp(-j / 100.0) + 1e-3
    if kind == "expk":                       # sigma_j = exp(-j/k)
        return np.exp(-j / float(k))
    if kind == "sqrtgap64":                  # sigma_j = j^-1/2, times 0.1 beyond j = 64
        s = j ** -0.5
        s[64:] *= 0.1
        return s
    if kind.startswith("logspace"):          # Sec. 5 types: logspace(0, -e, r)
        e = float(kind[len("logspace"):])
        return np.logspace(0.0, -e, r)
    raise ValueError(kind)


def _orthonormal_np(rng, rows, cols):
    G = rng.standard_normal((rows, cols))
    Q, R = np.linalg.qr(G)
    return Q * np.sign(np.diag(R))[None, :]


def make_matrix_np(m, n, sigma, noise=0.0, seed=0, dtype="float64", factors=False):
    """A = U diag(sigma) V^T (+ noise * N(0,1)) built in float64, stored as dtype.

    dtype "bfloat16" returns a float32 array holding bf16-representable values
    (round to nearest even), i.e. the stored bf16 matrix promoted to fp32.
    With factors=True the result is (A, U, V): the orthonormal factors the
    matrix was built from (float64).
    """
    sigma = np.asarray(sigma, dtype=np.float64)
    r = sigma.size
    rng = np.random.default_rng(seed)
    U = _orthonormal_np(rng, m, r)
    V = _orthonormal_np(rng, n, r)
    A = (U * sigma[None, :]) @ V.T
    if noise:
        A += noise * rng.standard_normal((m, n))
    if dtype in ("float64", np.float64):
        return (A, U, V) if factors else A
    A32 = A.astype(np.float32)
    if dtype in ("float32", np.float32):
        return (A32, U, V) if factors else A32
    if dtype == "bfloat16":
        b = A32.view(np.uint32).astype(np.uint64)
        b = ((b + np.uint64(0x7FFF) + ((b >> np.uint64(16)) & np.uint64(1)))
             >> np.uint64(16)) << np.uint64(16)
        Ab = b.astype(np.uint32).view(np.float32)
        return (Ab, U, V) if factors else Ab
    raise ValueError(dtype)


def low_rank_np(m, n, rank, seed=0, dtype="float64"):
    """A matrix of exact rank ``rank`` (in float64): G1 G2^T with Gaussian factors."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, rank)) @ rng.standard_normal((rank, n)) / np.sqrt(n)
    return A.astype(dtype)


def make_matrix_torch(m, n, sigma, noise=0.0, seed=0, dtype="float32", device="cuda",
                      chunk_rows=8192):
    """The same recipe with the large products on a device (large workloads).

    The Gaussian factors are drawn and orthonormalised (LAPACK QR) on the host
    with numpy; A = U diag(sigma) V^T and the noise are formed on ``device``
    with torch's seeded generator.  Values differ from ``make_matrix_np`` for
    the same seed.  Returns a contiguous row-major tensor.
    """
    import torch
    sigma = np.asarray(sigma, dtype=np.float64)
    r = sigma.size
    rng = np.random.default_rng(seed)
    cdtype = torch.float64 if dtype == "float64" else torch.float32
    U = torch.from_numpy(_orthonormal_np(rng, m, r) * sigma[None, :]).to(device, cdtype)
    V = torch.from_numpy(_orthonormal_np(rng, n, r)).to(device, cdtype)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    prev_tf32 = torch.backends.cuda.matmul.allow_tf32 if str(device).startswith("cuda") else None
    if prev_tf32 is not None:
        torch.backends.cuda.matmul.allow_tf32 = False
    try:
        tdtype = {"float32": torch.float32, "bfloat16": torch.bfloat16,
                  "float64": torch.float64}[dtype]
        A = torch.empty(m, n, dtype=tdtype, device=device)
        for i0 in range(0, m, chunk_rows):
            i1 = min(m, i0 + chunk_rows)
            blk = U[i0:i1] @ V.T
            if noise:
                blk.add_(torch.randn(i1 - i0, n, generator=g, device=device, dtype=cdtype),
                         alpha=noise)
            A[i0:i1].copy_(blk)
        del U, V
        return A
    finally:
        if prev_tf32 is not None:
            torch.backends.cuda.matmul.allow_tf32 = prev_tf32
