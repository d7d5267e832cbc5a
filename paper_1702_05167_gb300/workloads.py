"""Seeded synthetic device generators shared by the CUDA path, the tests and the benchmark.

This module only *describes* devices: it builds the tight-binding Hamiltonian H (CSR, complex128),
the contact site sets, the diagonal retarded/lesser contact self-energies and the energy grids.
It holds none of the selected-inversion arithmetic, so both the CUDA path and the CPU oracle can be
fed from it without sharing method code.

Conventions (Section 3.1, the cuboid device with a 7-point stencil and diagonal "SPARSE" self-energy):

* site (x, y, z) of an Nx x Ny x Nz grid has index s = (x*Ny + y)*Nz + z, so every x-plane is a
  contiguous block of Ny*Nz sites; x is the transport direction (contacts on x = 0 and x = Nx-1);
* unknown u = s*orb + o for orbital o of site s;
* A(E) = (E + i*eta) I - H - Sigma^r  (Eq. 1 with the usual infinitesimal eta);
* wide-band contacts: Sigma^r = -i*Gamma/2 on every contact unknown, Sigma^< = i*f*Gamma (Eq. 2).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Device:
    """A tight-binding device: H in CSR over unknowns plus its contacts."""

    dims: tuple            # (Nx, Ny, Nz) sites per direction
    orb: int               # orbitals per site
    rowptr: np.ndarray     # int64 [n+1]
    col: np.ndarray        # int32 [nnz]
    val: np.ndarray        # complex128 [nnz]
    contact_ptr: np.ndarray    # int64 [n_contacts+1] into contact_sites
    contact_sites: np.ndarray  # int32 site indices, contact after contact
    gamma: np.ndarray          # float64 [n_contacts] broadening Gamma of each contact (eV)
    meta: dict = field(default_factory=dict)

    @property
    def n_sites(self) -> int:
        return int(np.prod(self.dims))

    @property
    def n(self) -> int:
        return self.n_sites * self.orb

    def contact_unknowns(self) -> np.ndarray:
        """Unknown indices of all contacts, contact after contact, site-major then orbital."""
        s = self.contact_sites.astype(np.int64)
        return (s[:, None] * self.orb + np.arange(self.orb)[None, :]).reshape(-1)

    def contact_of_unknown(self) -> np.ndarray:
        """Contact id for each entry of contact_unknowns()."""
        counts = np.diff(self.contact_ptr) * self.orb
        return np.repeat(np.arange(len(counts)), counts)

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col, self.rowptr), shape=(self.n, self.n))


def site_index(x, y, z, dims):
    Nx, Ny, Nz = dims
    return (x * Ny + y) * Nz + z


def face_sites(dims, x):
    """Sites of the plane at transport coordinate x, in increasing index order."""
    Nx, Ny, Nz = dims
    y, z = np.meshgrid(np.arange(Ny), np.arange(Nz), indexing="ij")
    return site_index(x, y.reshape(-1), z.reshape(-1), dims).astype(np.int32)


def _bonds(dims):
    """Nearest-neighbour bonds (s, s+step) along +x, +y, +z with their direction index."""
    Nx, Ny, Nz = dims
    idx = np.arange(Nx * Ny * Nz).reshape(Nx, Ny, Nz)
    out = []
    for d, sl in enumerate([(slice(0, Nx - 1), slice(None), slice(None)),
                            (slice(None), slice(0, Ny - 1), slice(None)),
                            (slice(None), slice(None), slice(0, Nz - 1))]):
        a = idx[sl].reshape(-1)
        step = [Ny * Nz, Nz, 1][d]
        out.append((a, a + step, d))
    return out


def _csr_from_blocks(n_sites, orb, diag_blocks, bond_list):
    """Assemble CSR over unknowns from per-site onsite blocks and per-bond hopping blocks.

    diag_blocks: [n_sites, orb, orb]; bond_list: list of (a_sites, b_sites, blocks[orb,orb] or
    [nb,orb,orb]) where H[a,b] = block and H[b,a] = block^T.
    """
    import scipy.sparse as sp
    rows, cols, vals = [], [], []
    o = np.arange(orb)
    # onsite blocks
    s = np.arange(n_sites)
    r = (s[:, None, None] * orb + o[None, :, None]) + 0 * o[None, None, :]
    c = (s[:, None, None] * orb + o[None, None, :]) + 0 * o[None, :, None]
    rows.append(r.reshape(-1)); cols.append(c.reshape(-1)); vals.append(diag_blocks.reshape(-1))
    for a, b, blk in bond_list:
        blk = np.broadcast_to(blk, (len(a), orb, orb))
        r = a[:, None, None] * orb + o[None, :, None] + 0 * o[None, None, :]
        c = b[:, None, None] * orb + o[None, None, :] + 0 * o[None, :, None]
        rows += [r.reshape(-1), c.transpose(0, 2, 1).reshape(-1)]
        cols += [c.reshape(-1), r.transpose(0, 2, 1).reshape(-1)]
        vals += [blk.reshape(-1), blk.transpose(0, 2, 1).reshape(-1)]
    n = n_sites * orb
    M = sp.coo_matrix((np.concatenate(vals).astype(np.complex128),
                       (np.concatenate(rows), np.concatenate(cols))), shape=(n, n)).tocsr()
    M.sum_duplicates()
    M.sort_indices()
    return (M.indptr.astype(np.int64), M.indices.astype(np.int32), M.data.astype(np.complex128))


def cubic_device(dims, t=-1.0, W=1.0, seed=0, gamma=0.5):
    """Single-orbital simple-cubic tight-binding grid (Section 3.1, 7-point stencil).

    Onsite energies uniform in [-W/2, W/2] from numpy's PCG64 with `seed`, hopping t between nearest
    neighbours, wide-band contacts with broadening `gamma` on faces x = 0 and x = Nx-1.
    """
    dims = tuple(int(d) for d in dims)
    rng = np.random.default_rng(seed)
    n_sites = int(np.prod(dims))
    eps = rng.uniform(-W / 2, W / 2, size=n_sites)
    diag = eps.reshape(n_sites, 1, 1).astype(np.complex128)
    bonds = [(a, b, np.full((1, 1), t, dtype=np.complex128)) for a, b, _ in _bonds(dims)]
    rowptr, col, val = _csr_from_blocks(n_sites, 1, diag, bonds)
    left, right = face_sites(dims, 0), face_sites(dims, dims[0] - 1)
    return Device(dims=dims, orb=1, rowptr=rowptr, col=col, val=val,
                  contact_ptr=np.array([0, len(left), len(left) + len(right)], dtype=np.int64),
                  contact_sites=np.concatenate([left, right]).astype(np.int32),
                  gamma=np.array([gamma, gamma]),
                  meta=dict(kind="cubic", t=t, W=W, seed=seed, onsite=eps))


def magnetic_cubic_device(dims, phi, t=-1.0, W=1.0, seed=0, gamma=0.5):
    """cubic_device in a uniform magnetic field along z: Peierls phases in the Landau gauge
    A = (0, B x, 0), so the hopping from (x, y, z) to (x, y+1, z) is t exp(2 pi i phi x) (phi: flux
    per plaquette in flux quanta) and the reverse hopping its conjugate. H is Hermitian and, unless
    2 phi is an integer, not symmetric. Onsite energies and contacts as cubic_device(dims, t, W,
    seed, gamma)."""
    import scipy.sparse as sp
    base = cubic_device(dims, t=t, W=W, seed=seed, gamma=gamma)
    Nx, Ny, Nz = base.dims
    H = base.to_scipy().tolil()
    for x in range(Nx):
        ph = t * np.exp(2j * np.pi * phi * x)
        for y in range(Ny - 1):
            for z in range(Nz):
                a, b = site_index(x, y, z, base.dims), site_index(x, y + 1, z, base.dims)
                H[a, b] = ph
                H[b, a] = np.conj(ph)
    M = sp.csr_matrix(H)
    M.sort_indices()
    return Device(dims=base.dims, orb=1, rowptr=M.indptr.astype(np.int64), col=M.indices.astype(np.int32),
                  val=M.data.astype(np.complex128), contact_ptr=base.contact_ptr,
                  contact_sites=base.contact_sites, gamma=base.gamma,
                  meta=dict(base.meta, kind="magnetic", phi=phi))


def gbng_device(nx, ny, nz, t=-2.7, t_perp=0.35, delta_bn=2.0, W=0.0, seed=0, gamma=1.0):
    """Synthetic stand-in for the graphene - hBN - graphene stack of Section 3.2 (p_z orbitals).

    nz honeycomb layers of nx x ny sites, each in brick-wall form: bonds (x, y)-(x+1, y), and
    (x, y)-(x, y+1) where x + y + z is even (three in-plane neighbours in the bulk). The outer two
    layers are graphene (onsite 0), the inner ones hBN (onsite +delta_bn on the x + y + z even
    sublattice, -delta_bn on the other). AB (Bernal) stacking: site (x, y, z) couples to
    (x, y, z+1) with t_perp where x + y + z is even, so half the sites of a layer have a partner in
    each neighbouring layer. Onsite disorder uniform in [-W/2, W/2]. Contacts (wide-band,
    broadening gamma): the top layer's row y = 0 and the bottom layer's row y = ny-1, where the
    paper's semi-infinite ribbon electrodes attach. Sites are numbered (y * nz + z) * nx + x, so
    grid_dims (ny, nz, nx) describe the same grid and the y-slices are RGF layers.
    Parameters are synthetic choices (the paper takes them from its reference).
    """
    import scipy.sparse as sp
    rng = np.random.default_rng(seed)
    dims = (int(ny), int(nz), int(nx))
    n = ny * nz * nx
    idx = lambda x, y, z: (y * nz + z) * nx + x
    rows, cols, vals = [], [], []
    def bond(a, b, v):
        rows.extend([a, b]); cols.extend([b, a]); vals.extend([v, v])
    eps = rng.uniform(-W / 2, W / 2, size=n) if W > 0 else np.zeros(n)
    for z in range(nz):
        bn = 0 < z < nz - 1
        for y in range(ny):
            for x in range(nx):
                a = idx(x, y, z)
                if bn:
                    eps[a] += delta_bn if (x + y + z) % 2 == 0 else -delta_bn
                if x + 1 < nx:
                    bond(a, idx(x + 1, y, z), t)
                if y + 1 < ny and (x + y + z) % 2 == 0:
                    bond(a, idx(x, y + 1, z), t)
                if z + 1 < nz and (x + y + z) % 2 == 0:
                    bond(a, idx(x, y, z + 1), t_perp)
    rows.extend(range(n)); cols.extend(range(n)); vals.extend(eps.tolist())
    M = sp.coo_matrix((np.asarray(vals, dtype=np.complex128), (rows, cols)), shape=(n, n)).tocsr()
    M.sum_duplicates()
    M.sort_indices()
    left = np.array([idx(x, 0, nz - 1) for x in range(nx)], dtype=np.int32)
    right = np.array([idx(x, ny - 1, 0) for x in range(nx)], dtype=np.int32)
    return Device(dims=dims, orb=1, rowptr=M.indptr.astype(np.int64), col=M.indices.astype(np.int32),
                  val=M.data.astype(np.complex128),
                  contact_ptr=np.array([0, nx, 2 * nx], dtype=np.int64),
                  contact_sites=np.concatenate([left, right]).astype(np.int32),
                  gamma=np.array([gamma, gamma]), meta=dict(kind="gbng", onsite=eps))


def wire_device(dims, orb=10, seed=0, onsite_range=8.0, hop_fro=2.0, gamma=0.6):
    """Multi-orbital wire: random real-symmetric onsite blocks Q diag(U[-r, r]) Q^T per site and one
    random hopping block per bond direction scaled to Frobenius norm `hop_fro` (reverse bond gets the
    transpose), contacts on the x = 0 and x = Nx-1 planes."""
    dims = tuple(int(d) for d in dims)
    rng = np.random.default_rng(seed)
    n_sites = int(np.prod(dims))
    diag = np.empty((n_sites, orb, orb))
    for s in range(n_sites):
        q, _ = np.linalg.qr(rng.standard_normal((orb, orb)))
        diag[s] = (q * rng.uniform(-onsite_range, onsite_range, size=orb)) @ q.T
    diag = 0.5 * (diag + diag.transpose(0, 2, 1))
    bonds = []
    for a, b, d in _bonds(dims):
        blk = rng.standard_normal((orb, orb))
        blk *= hop_fro / np.linalg.norm(blk)
        bonds.append((a, b, blk.astype(np.complex128)))
    rowptr, col, val = _csr_from_blocks(n_sites, orb, diag.astype(np.complex128), bonds)
    left, right = face_sites(dims, 0), face_sites(dims, dims[0] - 1)
    return Device(dims=dims, orb=orb, rowptr=rowptr, col=col, val=val,
                  contact_ptr=np.array([0, len(left), len(left) + len(right)], dtype=np.int64),
                  contact_sites=np.concatenate([left, right]).astype(np.int32),
                  gamma=np.array([gamma, gamma]), meta=dict(kind="wire", seed=seed))


def chain_device(N, t=-1.0, eps=None, gamma=0.5):
    """1D chain of N sites (grid N x 1 x 1) with end contacts: the closed-form test case."""
    eps = np.zeros(N) if eps is None else np.asarray(eps, dtype=float)
    diag = eps.reshape(N, 1, 1).astype(np.complex128)
    a = np.arange(N - 1)
    rowptr, col, val = _csr_from_blocks(N, 1, diag, [(a, a + 1, np.full((1, 1), t, np.complex128))])
    return Device(dims=(N, 1, 1), orb=1, rowptr=rowptr, col=col, val=val,
                  contact_ptr=np.array([0, 1, 2], dtype=np.int64),
                  contact_sites=np.array([0, N - 1], dtype=np.int32),
                  gamma=np.array([gamma, gamma]), meta=dict(kind="chain", t=t, onsite=eps))


def with_scattering_contact(dev: Device) -> Device:
    """Copy of dev with one more contact holding every site outside its contacts, broadening 0: the
    scattering region, so that every unknown has a self-energy slot."""
    inside = np.zeros(dev.n_sites, dtype=bool)
    inside[dev.contact_sites] = True
    rest = np.nonzero(~inside)[0].astype(np.int32)
    ptr = np.append(dev.contact_ptr, dev.contact_ptr[-1] + len(rest)).astype(np.int64)
    return Device(dims=dev.dims, orb=dev.orb, rowptr=dev.rowptr, col=dev.col, val=dev.val,
                  contact_ptr=ptr, contact_sites=np.concatenate([dev.contact_sites, rest]),
                  gamma=np.append(dev.gamma, 0.0), meta=dict(dev.meta, scattering_contact=True))


def cubic_lead(dims, t=-1.0):
    """Clean semi-infinite lead continuing a cubic device along x: the layer Hamiltonian H00 (the
    Ny x Nz cross-section, onsite 0, hopping t) and the coupling H01 from one layer to the next
    (t on every site). Face-local site order y * Nz + z, as face_sites."""
    _, Ny, Nz = (int(d) for d in dims)
    m = Ny * Nz
    H00 = np.zeros((m, m), dtype=np.complex128)
    for y in range(Ny):
        for z in range(Nz):
            a = y * Nz + z
            if y + 1 < Ny:
                H00[a, a + Nz] = H00[a + Nz, a] = t
            if z + 1 < Nz:
                H00[a, a + 1] = H00[a + 1, a] = t
    return H00, t * np.eye(m, dtype=np.complex128)


def self_energies(dev: Device, n_E: int, f=(1.0, 0.0)):
    """Diagonal wide-band self-energies over dev.contact_unknowns() for n_E energies.

    Sigma^r = -i Gamma_c / 2 and Sigma^< = i f_c Gamma_c on every unknown of contact c (energy
    independent in the wide-band limit, repeated per energy so that callers may vary them).
    Returns (sigma_r, sigma_less), each complex128 [n_E, n_contact_unknowns].
    """
    cid = dev.contact_of_unknown()
    g = dev.gamma[cid]
    fl = np.asarray(f, dtype=float)[cid]
    sr = np.broadcast_to(-0.5j * g, (n_E, len(cid))).astype(np.complex128)
    sl = np.broadcast_to(1j * fl * g, (n_E, len(cid))).astype(np.complex128)
    return np.ascontiguousarray(sr), np.ascontiguousarray(sl)


def plane_pairs(dev: Device, x):
    """All unknown pairs (u, v) coupling plane x to plane x+1 through one bond (same y, z, orbital
    pairs o, o'), i.e. the G^r coupling block between the two planes used for the current."""
    Nx, Ny, Nz = dev.dims
    a = face_sites(dev.dims, x).astype(np.int64)
    b = a + Ny * Nz
    o = np.arange(dev.orb)
    u = (a[:, None, None] * dev.orb + o[None, :, None] + 0 * o[None, None, :]).reshape(-1)
    v = (b[:, None, None] * dev.orb + o[None, None, :] + 0 * o[None, :, None]).reshape(-1)
    return np.stack([u, v], axis=1).astype(np.int32)


# ---- named workloads (seeded, synthetic) -------------------------------------------------------

def tiny():
    """8x8x8 grid, t=-1, onsite U[-0.5,0.5] seed 0, Gamma=0.5 on x=0 and x=7, eta=1e-6, E=0.3,
    f_L=1, f_R=0, leaves <= 4 per dimension."""
    dev = cubic_device((8, 8, 8), t=-1.0, W=1.0, seed=0, gamma=0.5)
    return dict(name="cubic_8x8x8_1E", dev=dev, energies=np.array([0.3]), eta=1e-6, leaf=4,
                f=(1.0, 0.0))


def mid(n_E=64):
    """32x32x32 grid, W=1.0, Gamma=0.5 contacts on x=0 and x=31, 64 energies in [-5.5, 5.5],
    eta=1e-6, leaves <= 8 per dimension, coupling pairs between planes x=15 and x=16."""
    dev = cubic_device((32, 32, 32), t=-1.0, W=1.0, seed=0, gamma=0.5)
    return dict(name="cubic_32x32x32_64E", dev=dev, energies=np.linspace(-5.5, 5.5, n_E),
                eta=1e-6, leaf=8, f=(1.0, 0.0), pairs=plane_pairs(dev, 15))


BATCH_DIMS = [(24, 24, 24), (32, 24, 24), (32, 32, 24), (40, 32, 32),
              (48, 32, 32), (24, 48, 16), (36, 36, 36), (48, 24, 40)]


def batching(n_E_total=256):
    """Eight cuboids with uneven separators, seeds 1000+k, energies linspace(-6, 6, 256) dealt out
    32 per cuboid (round robin)."""
    E = np.linspace(-6.0, 6.0, n_E_total)
    out = []
    for k, d in enumerate(BATCH_DIMS):
        dev = cubic_device(d, t=-1.0, W=1.0, seed=1000 + k, gamma=0.5)
        out.append(dict(name=f"cubic_{d[0]}x{d[1]}x{d[2]}", dev=dev, energies=E[k::len(BATCH_DIMS)],
                        eta=1e-6, leaf=8, f=(1.0, 0.0)))
    return out


def wire(n_E=128):
    """10-orbital wire on 64 x 12 x 12 sites (92160 unknowns), 128 energies in [-2, 2]."""
    dev = wire_device((64, 12, 12), orb=10, seed=0, gamma=0.6)
    return dict(name="wire_64x12x12_10orb", dev=dev, energies=np.linspace(-2.0, 2.0, n_E),
                eta=1e-6, leaf=8, f=(1.0, 0.0))
