"""Seeded synthetic inputs shaped like the paper's experiments.

This module holds no step of the decomposition method; it only builds test
matrices and random sketching matrices, and is shared by the tests, the
oracle runs and the benchmark.  Random draws use numpy's PCG64
(``numpy.random.default_rng``), which gives the same numbers on every
platform.

Spectrum matrices follow Section 6: A = U_a diag(sigma) V_a^T with U_a, V_a
random orthonormal factors (QR of N(0, 1) matrices with the sign of R's
diagonal fixed positive, i.e. Haar-distributed).
"""
import numpy as np
import torch

BASE_SEED = 1412


def rng(seed):
    return np.random.default_rng(seed)


def haar(m, r, g, device="cpu"):
    """m x r matrix with orthonormal columns, Haar-distributed (numpy's
    Householder QR on the host, then moved to ``device``)."""
    Q, R = np.linalg.qr(g.standard_normal((m, r)))
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return torch.from_numpy(Q * s).to(device)


def spectrum_matrix(m, n, sigma, seed, dtype=torch.float64, device="cpu"):
    """A = U_a diag(sigma) V_a^T, float64 arithmetic, cast once to ``dtype``.
    ``sigma`` has length r <= min(m, n); the remaining singular values are 0.
    Returns a contiguous row-major (m, n) tensor on ``device``."""
    sigma = np.asarray(sigma, dtype=np.float64)
    r = sigma.size
    g = rng(seed)
    Ua = haar(m, r, g, device)
    Va = haar(n, r, g, device)
    s = torch.from_numpy(sigma).to(device)
    A = (Ua * s) @ Va.T
    return A.to(dtype).contiguous()


def exp_decay(r, scale=10.0):
    """sigma_j = exp(-j / scale), j = 1..r."""
    return np.exp(-np.arange(1, r + 1) / scale)


def power_decay(r, power=2.0):
    """sigma_j = j^(-power), j = 1..r."""
    return np.arange(1, r + 1, dtype=np.float64) ** (-power)


def logspaced(r, lo_exp):
    """sigma logspaced from 1 to 10^lo_exp (Set 1/2 of Section 6)."""
    return np.logspace(0, lo_exp, r)


def gaussian(rows, cols, seed, dtype=torch.float64, device="cpu"):
    """i.i.d. N(0, 1) matrix (the test matrix Omega of Algorithm 4)."""
    G = rng(seed).standard_normal((rows, cols))
    return torch.from_numpy(G).to(dtype).to(device).contiguous()


def planted_pivots(m, n, k, seed, decay=2.0 ** -0.5, offdiag=0.3,
                   dtype=torch.float64, device="cpu"):
    """Matrix whose column-pivoted QR order is fixed by construction:
    A = Q S P^T with Q Haar (m x r), S upper trapezoidal (r x n) with
    S(j, j) = decay^j and every off-diagonal entry of column l bounded by
    offdiag * S(j, j) / sqrt(n) for the rows j < its diagonal, and a random
    permutation P.  For r = min(m, n) >= k the first k pivots are
    P's first k columns, with norm gaps far above rounding.
    Returns (A, planted J)."""
    g = rng(seed)
    r = min(m, n)
    Q = haar(m, r, g).numpy()
    S = np.zeros((r, n))
    d = decay ** np.arange(r)
    for c in range(n):
        top = min(c, r)
        # rows above the diagonal: small relative to the smallest earlier
        # diagonal so each later column stays below its pivot's norm
        S[:top, c] = g.uniform(-1, 1, top) * offdiag * d[:top] / np.sqrt(n)
        if c < r:
            S[c, c] = d[c]
        else:
            # columns beyond r: norm below the last diagonal entry
            S[:r, c] = g.uniform(-1, 1, r) * offdiag * d[r - 1] / np.sqrt(n)
    perm = g.permutation(n)
    A = np.zeros((m, n))
    A[:, perm] = Q @ S
    return (torch.from_numpy(A).to(dtype).to(device).contiguous(),
            perm.astype(np.int64))


def exact_rank(m, n, k, seed, dtype=torch.float64, device="cpu"):
    """Exactly rank-k matrix X Y with Gaussian X (m x k), Y (k x n)."""
    g = rng(seed)
    X = g.standard_normal((m, k))
    Y = g.standard_normal((k, n))
    return torch.from_numpy(X @ Y).to(dtype).to(device).contiguous()


def laplace_block(m, n, seed, dtype=torch.float64, device="cpu"):
    """Laplace kernel block K(x, y) = 1 / |x - y| between m target points
    uniform in the unit box centred at the origin and n source points in the
    unit box centred at (3, 0, 0)."""
    g = rng(seed)
    x = g.uniform(-0.5, 0.5, (m, 3))
    y = g.uniform(-0.5, 0.5, (n, 3)) + np.array([3.0, 0.0, 0.0])
    d = np.sqrt(((x[:, None, :] - y[None, :, :]) ** 2).sum(-1))
    return torch.from_numpy(1.0 / d).to(dtype).to(device).contiguous()


def decay_with_floor(m, n, r, top_exp, floor, seed, device="cpu", dtype=torch.bfloat16):
    """A = U_a diag(sigma) V_a^T + floor * N / sqrt(n), sigma_j = 10^(top_exp j / r)
    for j <= r (top_exp < 0), U_a, V_a Haar (m x r, n x r), N i.i.d. N(0, 1)
    drawn on ``device`` from a generator seeded with ``seed``; computed in
    float32 and rounded once to ``dtype``.  The floor term stands for the
    singular values 10^-7 beyond r (its rounding to bfloat16 is far below the
    storage resolution of the leading part)."""
    g = rng(seed)
    sigma = 10.0 ** (top_exp * np.arange(1, r + 1) / r)
    Ua = haar(m, r, g, device).to(torch.float32)
    Va = haar(n, r, g, device).to(torch.float32)
    s = torch.from_numpy(sigma).to(torch.float32).to(device)
    A = (Ua * s) @ Va.T
    if floor > 0:
        gen = torch.Generator(device=device)
        gen.manual_seed(int(seed))
        A += floor / np.sqrt(n) * torch.randn(m, n, generator=gen, device=device,
                                              dtype=torch.float32)
    return A.to(dtype).contiguous()


def laplace_batch_shapes(nb, seed, lo=64, hi=512):
    """Block shapes (m_b, n_b), each uniform on {lo..hi}."""
    g = rng(seed)
    return [(int(a), int(b)) for a, b in g.integers(lo, hi + 1, size=(nb, 2))]


def laplace_batch(nb, seed, dtype=torch.float64, device="cpu", lo=64, hi=512):
    """nb Laplace blocks with m_b, n_b uniform on {lo..hi}; block b uses
    seed (seed, b) for its point clusters.  Returns (flat, shapes, offsets):
    the blocks stored row-major back to back in one tensor, each starting
    on a 16-byte boundary."""
    shapes = laplace_batch_shapes(nb, seed, lo, hi)
    esz = torch.empty((), dtype=dtype).element_size()
    align = max(1, 16 // esz)
    offsets, total = [], 0
    for m, n in shapes:
        offsets.append(total)
        total += (m * n + align - 1) // align * align
    flat = torch.zeros(total, dtype=dtype)
    for b, (m, n) in enumerate(shapes):
        blk = laplace_block(m, n, int(np.random.SeedSequence([seed, b]).generate_state(1)[0]),
                            dtype)
        flat[offsets[b]:offsets[b] + m * n] = blk.reshape(-1)
    return flat.to(device), shapes, offsets


# Named workloads -----------------------------------------------------------

def workload_small_f64(seed=BASE_SEED + 0, device="cpu"):
    """Dense FP64 400 x 300, sigma_j = exp(-j/10), deterministic, k = 40."""
    A = spectrum_matrix(400, 300, exp_decay(300), seed, torch.float64, device)
    return dict(A=A, k=40, p=-1, q=0, name="det_f64_400x300_k40")


def workload_mixed_bf16(seed=BASE_SEED + 2, device="cpu", m=20000, n=20000, k=500, p=20,
                        q=2):
    """BF16 20000 x 20000, sigma_j = 10^(-6j/500) for j <= 500, floor 1e-7,
    k = 500, p = 20, q = 2."""
    A = decay_with_floor(m, n, k, -6.0, 1e-7, seed, device)
    return dict(A=A, k=k, p=p, q=q, name=f"mixed_bf16_{m}x{n}_k{k}_p{p}_q{q}")


def workload_rand_f32(seed=BASE_SEED + 1, device="cpu", m=8000, n=6000,
                      k=200, p=10, q=1):
    """Dense FP32 8000 x 6000, sigma_j = j^-2, k = 200, p = 10, q = 1, with
    a Gaussian Omega of shape (k+p) x m."""
    A = spectrum_matrix(m, n, power_decay(min(m, n)), seed, torch.float32,
                        device)
    Om = gaussian(k + p, m, seed + 1000, torch.float32, device)
    return dict(A=A, Omega=Om, k=k, p=p, q=q,
                name=f"rand_f32_{m}x{n}_k{k}_p{p}_q{q}")


def sparse_rank_sum(m, n, coeffs, seed, dx=0.002, dy=0.02):
    """Sum of sparse rank-one terms, sum_j coeffs[j] x_j y_j^T, with x_j (m)
    and y_j (n) sparse and non-negative: round(dx m) and round(dy n) entries
    (at least one) at distinct random positions, values uniform on (0, 1].
    The shape of the test matrices A_1, A_2 of Section 6 (m = 300000,
    n = 300, 300 terms; the paper does not give the densities).  Returns a
    scipy.sparse CSR matrix (float64, sorted indices, duplicates summed)."""
    import scipy.sparse
    g = rng(seed)
    nx = max(1, int(round(dx * m)))
    ny = max(1, int(round(dy * n)))
    rows, cols, vals = [], [], []
    for c in coeffs:
        xi = g.choice(m, nx, replace=False)
        xv = 1.0 - g.random(nx)
        yi = g.choice(n, ny, replace=False)
        yv = 1.0 - g.random(ny)
        rows.append(np.repeat(xi, ny))
        cols.append(np.tile(yi, nx))
        vals.append(c * np.outer(xv, yv).ravel())
    A = scipy.sparse.coo_matrix((np.concatenate(vals), (np.concatenate(rows),
                                                        np.concatenate(cols))), shape=(m, n))
    A = A.tocsr()
    A.sum_duplicates()
    A.sort_indices()
    return A


def a1_coeffs(terms=300, big=2.0, lead=10):
    """Coefficients of A_1 (big = 2) and A_2 (big = 1000) in Section 6:
    big / j for j <= lead, 1 / j after."""
    j = np.arange(1, terms + 1, dtype=np.float64)
    return np.where(j <= lead, big / j, 1.0 / j)


def to_torch_csr(A, dtype=torch.float64, device="cpu"):
    """scipy CSR -> torch sparse CSR tensor (values cast once to dtype)."""
    return torch.sparse_csr_tensor(torch.from_numpy(A.indptr.astype(np.int64)),
                                   torch.from_numpy(A.indices.astype(np.int64)),
                                   torch.from_numpy(A.data).to(dtype), size=A.shape,
                                   device=device, check_invariants=True)
