"""Independent references used to pin the oracle (test side only).

Nothing here calls the oracle.  It provides
  * dense Hamiltonians built from Kronecker products of 2x2 Pauli matrices,
    written from the paper's definitions (Sec. III), for exact
    diagonalisation and exact <H>;
  * the Jordan-Wigner closed form of the open TFIM ground energy: minus the
    sum of the singular values of the N x N bidiagonal matrix with h on the
    diagonal and J on the superdiagonal;
  * a log Psi built on the library GRU cell (torch's gru_cell), so the
    paper's GRU (App. A) is checked against a third-party implementation
    through the mapping u = 1 - z_torch, r = r_torch, W_h <-> W_hn.
"""
import itertools

import numpy as np
import torch

SX = np.array([[0, 1], [1, 0]], dtype=np.complex128)
SY = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
SZ = np.array([[1, 0], [0, -1]], dtype=np.complex128)
I2 = np.eye(2, dtype=np.complex128)
PAULI = {"X": SX, "Y": SY, "Z": SZ}


def all_configs(N):
    """Basis order: configuration sigma <-> index b with sigma_0 the most
    significant bit (the order of np.kron)."""
    return np.array(list(itertools.product([0, 1], repeat=N)), dtype=np.uint8)


def pauli_string(N, ops):
    mats = [I2] * N
    for k, p in ops:
        mats[k] = PAULI[p] @ mats[k]
    out = mats[0]
    for m in mats[1:]:
        out = np.kron(out, m)
    return out


def zigzag(Lx, Ly):
    """Lattice coordinates (i, j) -> path index k of the zig-zag path."""
    idx = {}
    for j in range(Ly):
        for i in range(Lx):
            idx[(i, j)] = j * Lx + (i if j % 2 == 0 else Lx - 1 - i)
    return idx


def dense_tfim(N, J=1.0, h=1.0):
    H = np.zeros((2 ** N, 2 ** N), dtype=np.complex128)
    for i in range(N - 1):
        H -= J * pauli_string(N, [(i, "Z"), (i + 1, "Z")])
    for i in range(N):
        H -= h * pauli_string(N, [(i, "X")])
    return H


def dense_cluster_zxz(N):
    H = np.zeros((2 ** N, 2 ** N), dtype=np.complex128)
    for i in range(1, N - 1):
        H -= pauli_string(N, [(i - 1, "Z"), (i, "X"), (i + 1, "Z")])
    return H


def dense_cluster_paper(N):
    """Sec. III.B, 1-indexed sites 1..N."""
    H = np.zeros((2 ** N, 2 ** N), dtype=np.complex128)
    s = lambda k: k - 1  # 1-indexed -> 0-indexed
    for k in range(2, N - 1):
        H -= pauli_string(N, [(s(k - 1), "X"), (s(k), "Z"), (s(k + 1), "X")])
    H -= pauli_string(N, [(s(1), "Z"), (s(2), "X")])
    H -= pauli_string(N, [(s(N - 1), "X"), (s(N), "X")])
    H -= pauli_string(N, [(s(N - 2), "X"), (s(N - 1), "Z"), (s(N), "Z")])
    return H


def dense_j1j2(Lx, Ly, J1=1.0, J2=0.0):
    """sum over bonds of J/4 (XX + YY + ZZ) = J S_i.S_j, open lattice."""
    N = Lx * Ly
    idx = zigzag(Lx, Ly)
    H = np.zeros((2 ** N, 2 ** N), dtype=np.complex128)
    for (i, j), k in idx.items():
        nbrs = [((i + 1, j), J1), ((i, j + 1), J1),
                ((i + 1, j + 1), J2), ((i + 1, j - 1), J2)]
        for c, J in nbrs:
            if c in idx and J != 0.0:
                q = idx[c]
                for p in "XYZ":
                    H += (J / 4.0) * pauli_string(N, [(k, p), (q, p)])
    return H


def tfim_jw_energy(N, J=1.0, h=1.0):
    B = np.diag(np.full(N, h)) + np.diag(np.full(N - 1, J), 1)
    return -np.sum(np.linalg.svd(B, compute_uv=False))


# ------------------------------------------------ torch GRU-cell log psi
def split_theta(theta, spec):
    """Views of the flat parameter vector in layout order."""
    dh = spec.dh
    din = 4 if spec.dim == 2 else 2
    shapes = []
    if spec.dim == 2:
        shapes += [("U1", (dh, dh)), ("U2", (dh, dh))]
    shapes += [("Wu", (dh, dh + din)), ("bu", (dh,)), ("Wr", (dh, dh + din)),
               ("br", (dh,)), ("Wh", (dh, dh)), ("bh", (dh,)),
               ("Win", (dh, din)), ("bin", (dh,)), ("U", (2, dh)), ("c", (2,))]
    if spec.cplx:
        shapes += [("Uphi", (2, dh)), ("cphi", (2,))]
    out, o = {}, 0
    for name, shp in shapes:
        n = int(np.prod(shp))
        out[name] = theta[o:o + n].reshape(shp)
        o += n
    assert o == theta.shape[0]
    return out


def torch_logpsi(spec, theta, spins):
    """log Psi(sigma) for each row of spins via torch's gru_cell (fp64).
    theta: torch tensor (may require grad).  Returns (re, im) tensors."""
    P = split_theta(theta, spec)
    dh = spec.dh
    din = 4 if spec.dim == 2 else 2
    # torch gate order (r, z, n); z = 1 - u  <=>  z = sigmoid(-(W_u [h;x] + b_u))
    w_ih = torch.cat([P["Wr"][:, dh:], -P["Wu"][:, dh:], P["Win"]], 0)
    w_hh = torch.cat([P["Wr"][:, :dh], -P["Wu"][:, :dh], P["Wh"]], 0)
    b_ih = torch.cat([P["br"], -P["bu"], P["bin"]], 0)
    b_hh = torch.cat([torch.zeros_like(P["br"]), torch.zeros_like(P["bu"]), P["bh"]], 0)
    sp = torch.as_tensor(np.asarray(spins), dtype=torch.long)
    B, N = sp.shape
    Lx, Ly = spec.Lx, spec.Ly
    if spec.dim == 2:
        idx = zigzag(Lx, Ly)
        coord = {k: c for c, k in idx.items()}
    hs = [None] * N
    logP = torch.zeros(B, dtype=torch.float64)
    phi = torch.zeros(B, dtype=torch.float64)
    nup = torch.zeros(B, dtype=torch.long)
    ndn = torch.zeros(B, dtype=torch.long)
    zero_h = torch.zeros(B, dh, dtype=torch.float64)
    onehot = torch.nn.functional.one_hot
    for k in range(N):
        x = torch.zeros(B, din, dtype=torch.float64)
        if spec.dim == 1:
            hp = hs[k - 1] if k > 0 else zero_h
            if k > 0:
                x = onehot(sp[:, k - 1], 2).double()
        else:
            i, j = coord[k]
            hc = (i - (-1) ** j, j)
            vc = (i, j - 1)
            hk = idx.get(hc)
            vk = idx.get(vc)
            h_hor = hs[hk] if hk is not None else zero_h
            h_ver = hs[vk] if vk is not None else zero_h
            hp = h_hor @ P["U1"].T + h_ver @ P["U2"].T
            parts = [onehot(sp[:, hk], 2).double() if hk is not None
                     else torch.zeros(B, 2, dtype=torch.float64),
                     onehot(sp[:, vk], 2).double() if vk is not None
                     else torch.zeros(B, 2, dtype=torch.float64)]
            x = torch.cat(parts, 1)
        h = torch._VF.gru_cell(x, hp, w_ih, w_hh, b_ih, b_hh)
        hs[k] = h
        z = h @ P["U"].T + P["c"]
        lp = torch.log_softmax(z, dim=1)
        lps = lp.gather(1, sp[:, k:k + 1]).squeeze(1)
        if spec.zmask:
            half = N // 2
            forced_dn = nup >= half
            forced_up = (ndn >= half) & ~forced_dn
            neg = torch.full_like(lps, -np.inf)
            lps = torch.where(forced_dn, torch.where(sp[:, k] == 1, torch.zeros_like(lps), neg), lps)
            lps = torch.where(forced_up, torch.where(sp[:, k] == 0, torch.zeros_like(lps), neg), lps)
        logP = logP + lps
        if spec.cplx:
            y = (h @ P["Uphi"].T + P["cphi"]).gather(1, sp[:, k:k + 1]).squeeze(1)
            phi = phi + np.pi * torch.nn.functional.softsign(y)
        nup = nup + (sp[:, k] == 0).long()
        ndn = ndn + (sp[:, k] == 1).long()
    im = phi
    if spec.marshall:
        idx = zigzag(Lx, Ly)
        onA = np.zeros(N, dtype=bool)
        for (i, j), k in idx.items():
            onA[k] = (i + j) % 2 == 1
        nA = (sp[:, torch.as_tensor(onA)] == 1).sum(1) % 2
        im = im + np.pi * nA.double()
    return 0.5 * logP, im
