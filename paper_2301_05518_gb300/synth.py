"""Seeded synthetic inputs: SU(3) gauge fields and staggered source vectors.

This module holds none of the smearing arithmetic.  It only draws inputs, and
both the CUDA library's tests/benchmarks and the CPU oracle receive exactly the
arrays it returns.  The paper measures on HISQ gauge configurations with point
and colour wall sources (Sec. 3, Sec. 4, Fig. 1); those configurations are not
available, so these generators stand in for them with the same structure:
SU(3) links, three-colour point/wall sources and many sources on one gauge
field.

Everything is built with torch on the requested device, slice by slice, from a
``torch.Generator`` seeded per (seed, t): a field drawn on one device is the
same whether it is drawn whole or a slice at a time, so the big lattices never
need a host copy.  Fields on different devices are different draws; a test that
feeds the oracle copies the device tensor to the host.

Shapes (complex128 unless ``dtype`` says otherwise):
    gauge  [Lt, Lz, Ly, Lx, nd, 3, 3], nd = 3 (x, y, z) or 4 (x, y, z, t)
    vecs   [nvec, Lt, Lz, Ly, Lx, 3]
``dims`` is always (Lx, Ly, Lz, Lt).
"""

from __future__ import annotations

import math

import torch

_GELL_MANN = None


def _gell_mann(device) -> torch.Tensor:
    """The eight Gell-Mann matrices, [8, 3, 3] complex128."""
    global _GELL_MANN
    if _GELL_MANN is None:
        g = torch.zeros(8, 3, 3, dtype=torch.complex128)
        g[0, 0, 1] = g[0, 1, 0] = 1
        g[1, 0, 1] = -1j
        g[1, 1, 0] = 1j
        g[2, 0, 0] = 1
        g[2, 1, 1] = -1
        g[3, 0, 2] = g[3, 2, 0] = 1
        g[4, 0, 2] = -1j
        g[4, 2, 0] = 1j
        g[5, 1, 2] = g[5, 2, 1] = 1
        g[6, 1, 2] = -1j
        g[6, 2, 1] = 1j
        g[7, 0, 0] = g[7, 1, 1] = 1 / math.sqrt(3)
        g[7, 2, 2] = -2 / math.sqrt(3)
        _GELL_MANN = g
    return _GELL_MANN.to(device)


def _gen(seed: int, t: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed((int(seed) * 1_000_003 + int(t) * 7919 + 12345) % (2 ** 63))
    return g


def _cnormal(shape, gen, device) -> torch.Tensor:
    """Complex Gaussian, real and imaginary parts iid N(0, 1)."""
    re = torch.randn(shape, generator=gen, device=device, dtype=torch.float64)
    im = torch.randn(shape, generator=gen, device=device, dtype=torch.float64)
    return torch.complex(re, im)


def reunitarize(m: torch.Tensor) -> torch.Tensor:
    """Project [..., 3, 3] onto SU(3): Gram-Schmidt on rows 1-2, row 3 = (r1 x r2)*.

    The determinant of the result is |r1 x r2|^2 = 1 up to rounding.
    """
    r1 = m[..., 0, :]
    r2 = m[..., 1, :]
    r1 = r1 / torch.linalg.vector_norm(r1, dim=-1, keepdim=True)
    proj = (r1.conj() * r2).sum(-1, keepdim=True)
    r2 = r2 - proj * r1
    r2 = r2 / torch.linalg.vector_norm(r2, dim=-1, keepdim=True)
    r3 = torch.stack([
        r1[..., 1] * r2[..., 2] - r1[..., 2] * r2[..., 1],
        r1[..., 2] * r2[..., 0] - r1[..., 0] * r2[..., 2],
        r1[..., 0] * r2[..., 1] - r1[..., 1] * r2[..., 0],
    ], dim=-1).conj()
    return torch.stack([r1, r2, r3], dim=-2)


def _expm_taylor(x: torch.Tensor, order: int = 18) -> torch.Tensor:
    """exp(x) for [..., 3, 3] by a Horner-form Taylor series (small ||x||)."""
    eye = torch.eye(3, dtype=x.dtype, device=x.device).expand_as(x)
    e = eye.clone()
    for k in range(order, 0, -1):
        e = eye + (x @ e) / k
    return e


def _slices(dims):
    Lx, Ly, Lz, Lt = dims
    return Lt, (Lz, Ly, Lx)


def gauge_near_unit(dims, eps: float, seed: int, nd: int = 4, device="cpu") -> torch.Tensor:
    """U = exp(i eps H), H = sum_a h_a lambda_a / 2, h_a ~ N(0, 1), projected to SU(3)."""
    Lt, sp = _slices(dims)
    lam = _gell_mann(device)
    out = torch.empty((Lt,) + sp + (nd, 3, 3), dtype=torch.complex128, device=device)
    for t in range(Lt):
        g = _gen(seed, t, device)
        h = torch.randn(sp + (nd, 8), generator=g, device=device, dtype=torch.float64)
        H = torch.einsum("...a,aij->...ij", h.to(torch.complex128), lam) * 0.5
        out[t] = reunitarize(_expm_taylor(1j * eps * H))
    return out


def gauge_haar(dims, seed: int, nd: int = 4, device="cpu") -> torch.Tensor:
    """Haar-random SU(3) links: Gram-Schmidt of two iid complex Gaussian rows."""
    Lt, sp = _slices(dims)
    out = torch.empty((Lt,) + sp + (nd, 3, 3), dtype=torch.complex128, device=device)
    for t in range(Lt):
        g = _gen(seed, t, device)
        out[t] = reunitarize(_cnormal(sp + (nd, 3, 3), g, device))
    return out


def gauge_unit(dims, nd: int = 4, device="cpu") -> torch.Tensor:
    """The free field U = 1."""
    Lx, Ly, Lz, Lt = dims
    eye = torch.eye(3, dtype=torch.complex128, device=device)
    return eye.expand(Lt, Lz, Ly, Lx, nd, 3, 3).contiguous()


def gauge_transform_haar(dims, seed: int, device="cpu") -> torch.Tensor:
    """One Haar-random SU(3) matrix G(x) per site, [Lt, Lz, Ly, Lx, 3, 3]."""
    return gauge_haar(dims, seed, nd=1, device=device)[..., 0, :, :]


def point_sources(dims, sites, colors, dtype=torch.complex128, device="cpu") -> torch.Tensor:
    """psi_v(x) = e_{colors[v]} at sites[v] = (x, y, z, t), zero elsewhere."""
    Lx, Ly, Lz, Lt = dims
    out = torch.zeros((len(sites), Lt, Lz, Ly, Lx, 3), dtype=dtype, device=device)
    for v, ((x, y, z, t), c) in enumerate(zip(sites, colors)):
        out[v, t, z, y, x, c] = 1
    return out


def corner_wall_sources(dims, t: int = 0, dtype=torch.complex128, device="cpu") -> torch.Tensor:
    """24 corner wall sources: vector v = 3 * corner + color.

    Corner c in 0..7 selects the sites of slice t with (x & 1, y & 1, z & 1) =
    (c & 1, (c >> 1) & 1, (c >> 2) & 1); there psi = e_color, zero elsewhere.
    """
    Lx, Ly, Lz, Lt = dims
    out = torch.zeros((24, Lt, Lz, Ly, Lx, 3), dtype=dtype, device=device)
    for c in range(8):
        bx, by, bz = c & 1, (c >> 1) & 1, (c >> 2) & 1
        for a in range(3):
            out[3 * c + a, t, bz::2, by::2, bx::2, a] = 1
    return out


def color_wall_sources(dims, t: int = 0, dtype=torch.complex128, device="cpu") -> torch.Tensor:
    """Three colour wall sources on slice t: psi_a(x) = e_a at every site of t."""
    Lx, Ly, Lz, Lt = dims
    out = torch.zeros((3, Lt, Lz, Ly, Lx, 3), dtype=dtype, device=device)
    for a in range(3):
        out[a, t, ..., a] = 1
    return out


def gaussian_vectors(dims, nvec: int, seed: int, dtype=torch.complex128, device="cpu",
                     t: int | None = None) -> torch.Tensor:
    """Gaussian color vectors, re and im iid N(0, 1); only slice t if given."""
    Lt, sp = _slices(dims)
    real = torch.float64 if dtype == torch.complex128 else torch.float32
    out = torch.zeros((nvec, Lt) + sp + (3,), dtype=dtype, device=device)
    ts = range(Lt) if t is None else [t]
    for tt in ts:
        g = _gen(seed, tt, device)
        re = torch.randn((nvec,) + sp + (3,), generator=g, device=device, dtype=torch.float64)
        im = torch.randn((nvec,) + sp + (3,), generator=g, device=device, dtype=torch.float64)
        out[:, tt] = torch.complex(re.to(real), im.to(real))
    return out


def as_real(z: torch.Tensor) -> torch.Tensor:
    """Complex tensor -> contiguous real view with a trailing [re, im] axis."""
    return torch.view_as_real(z.contiguous())
