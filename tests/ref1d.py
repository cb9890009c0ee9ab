"""Independent 1D constructions used to pin the oracle (tests only).

Everything here is 1D polynomial algebra in numpy: Gauss-Lobatto nodes as
roots of P'_{k-1} from numpy's Legendre class, Lagrange polynomials in
product form, 1D integrals with numpy's Gauss-Legendre rule on more points
than needed (so they are exact).  No code from the oracle is used, and the
3D operators are built from 1D pieces, so agreement with the oracle's
brute-force 3D quadrature is a second route, not a re-run.

The 3D Cartesian operators are assembled as sums of Kronecker products of
these 1D matrices, the separable form of the Remark in Sec. 2.1 of
Kronbichler & Kormann (L = L1 (x) M2 + M1 (x) L2).
"""
import numpy as np
from numpy.polynomial import legendre as L
from numpy.polynomial import polynomial as P


def gl_nodes(k):
    """Gauss-Lobatto nodes on [0,1]: 0, 1 and the roots of P'_{k-1}."""
    if k == 2:
        t = np.array([-1.0, 1.0])
    else:
        inner = np.sort(L.Legendre.basis(k - 1).deriv().roots().real)
        t = np.concatenate([[-1.0], inner, [1.0]])
    return 0.5 * (t + 1.0)


def lagrange_coeffs(nodes):
    """Monomial coefficients of the Lagrange polynomials on ``nodes``."""
    k = len(nodes)
    out = []
    for j in range(k):
        others = np.delete(nodes, j)
        c = P.polyfromroots(others)
        out.append(c / P.polyval(nodes[j], c))
    return out


def _lagrange_eval(nodes, j, t):
    """Value and derivative of Lagrange polynomial j at points t (product form)."""
    t = np.asarray(t, dtype=np.float64)
    others = np.delete(nodes, j)
    den = np.prod(nodes[j] - others)
    val = np.prod(t[..., None] - others, axis=-1) / den
    der = np.zeros_like(t)
    for l in range(len(others)):
        rest = np.delete(others, l)
        der = der + np.prod(t[..., None] - rest, axis=-1)
    return val, der / den


def matrices_1d(p):
    """Reference-interval mass M, stiffness K, convection C_ij = int l_i' l_j,
    and endpoint values/derivatives of the GL-Lagrange basis of degree p.
    Integrals use numpy's own Gauss-Legendre rule with p+3 points (exact for
    the degree-2p integrands), not the oracle's rule."""
    k = p + 1
    x = gl_nodes(k)
    tq, wq = L.leggauss(k + 2)
    tq, wq = 0.5 * (tq + 1.0), 0.5 * wq
    V = np.array([_lagrange_eval(x, j, tq)[0] for j in range(k)])
    D = np.array([_lagrange_eval(x, j, tq)[1] for j in range(k)])
    M = (V * wq) @ V.T
    K = (D * wq) @ D.T
    C = (D * wq) @ V.T
    ends = [np.array([_lagrange_eval(x, j, np.array(e))[i] for j in range(k)])
            for e in (0.0, 1.0) for i in (0, 1)]
    v0, d0, v1, d1 = ends
    return dict(M=M, K=K, C=C, v0=v0, v1=v1, d0=d0, d1=d1, x=x)


def global_mass(p, N):
    r = matrices_1d(p)
    return np.kron(np.eye(N), r["M"] / N)


def sipg_1d(p, N, periodic, penalty=None):
    """Global 1D SIPG matrix on N uniform cells of [0,1] (h = 1/N):
    sum_K int v'u' + sum_F [-{v'}[u] - [v]{u'} + tau [v][u]] with the mirror
    principle u+ = -u-, u+' = u-' at Dirichlet points; tau = (p+1)^2/h."""
    r = matrices_1d(p)
    k = p + 1
    h = 1.0 / N
    tau = (p + 1) ** 2 / h if penalty is None else penalty
    n = N * k
    A = np.zeros((n, n))
    for c in range(N):
        A[c * k:(c + 1) * k, c * k:(c + 1) * k] += r["K"] / h
    # trace vectors: value and derivative of cell c at its right (1) / left (0) end
    def val(c, end):
        e = np.zeros(n)
        e[c * k:(c + 1) * k] = r["v1"] if end else r["v0"]
        return e

    def der(c, end):
        e = np.zeros(n)
        e[c * k:(c + 1) * k] = (r["d1"] if end else r["d0"]) / h
        return e

    faces = range(N) if periodic else range(N - 1)
    for f in faces:  # face between cell f (left, "-") and f+1 (right, "+"), n = +1
        lc, rc = f, (f + 1) % N
        jump = val(lc, 1) - val(rc, 0)
        avg = 0.5 * (der(lc, 1) + der(rc, 0))
        A += -np.outer(avg, jump) - np.outer(jump, avg) + tau * np.outer(jump, jump)
    if not periodic:
        for c, end, sgn in ((0, 0, -1.0), (N - 1, 1, 1.0)):
            v = val(c, end)
            dn = sgn * der(c, end)
            A += -np.outer(dn, v) - np.outer(v, dn) + 2.0 * tau * np.outer(v, v)
    return A


def advection_1d(p, N, periodic, c):
    """Global 1D upwind advection matrix for constant speed c:
    -(v', c u) + (v- - v+)(c/2 (u- + u+) + |c|/2 (u- - u+)) on interior
    points, |c n| v u at Dirichlet points."""
    r = matrices_1d(p)
    k = p + 1
    n = N * k
    A = np.zeros((n, n))
    for e in range(N):
        A[e * k:(e + 1) * k, e * k:(e + 1) * k] -= c * r["C"]

    def val(e, end):
        v = np.zeros(n)
        v[e * k:(e + 1) * k] = r["v1"] if end else r["v0"]
        return v

    faces = range(N) if periodic else range(N - 1)
    for f in faces:
        lm, rp = val(f, 1), val((f + 1) % N, 0)
        A += np.outer(lm - rp, 0.5 * c * (lm + rp) + 0.5 * abs(c) * (lm - rp))
    if not periodic:
        for e, end in ((0, 0), (N - 1, 1)):
            v = val(e, end)
            A += abs(c) * np.outer(v, v)
    return A


def tensor_to_dof_permutation(p, Ns):
    """perm[t] = oracle dof index of tensor index t = gx + nx*(gy + ny*gz),
    where g_d = i_d * k + local index (x fastest).  Oracle numbering: cell
    c = ix + Nx (iy + Ny iz), dof c k^3 + i0 + k (i1 + k i2)."""
    k = p + 1
    Nx, Ny, Nz = Ns
    gx, gy, gz = np.meshgrid(np.arange(Nx * k), np.arange(Ny * k), np.arange(Nz * k), indexing="ij")
    gx, gy, gz = gx.transpose(2, 1, 0).ravel(), gy.transpose(2, 1, 0).ravel(), gz.transpose(2, 1, 0).ravel()
    ix, i0 = gx // k, gx % k
    iy, i1 = gy // k, gy % k
    iz, i2 = gz // k, gz % k
    cell = ix + Nx * (iy + Ny * iz)
    return cell * k ** 3 + i0 + k * (i1 + k * i2)


def kron3(Ax, Ay, Az):
    """Tensor operator with x fastest: (Az (x) Ay (x) Ax)."""
    return np.kron(Az, np.kron(Ay, Ax))


def to_dof_order(T, p, Ns):
    perm = tensor_to_dof_permutation(p, Ns)
    n = len(perm)
    D = np.zeros((n, n))
    D[np.ix_(perm, perm)] = T
    return D


def separable_sipg(p, Ns, periodic):
    Ms = [global_mass(p, N) for N in Ns]
    As = [sipg_1d(p, N, periodic) for N in Ns]
    T = kron3(As[0], Ms[1], Ms[2]) + kron3(Ms[0], As[1], Ms[2]) + kron3(Ms[0], Ms[1], As[2])
    return to_dof_order(T, p, Ns)


def separable_advection(p, Ns, periodic, c):
    Ms = [global_mass(p, N) for N in Ns]
    # the 1D pieces carry the cell-size scaling: convection and face terms are
    # h-independent in 1D, mass is h-scaled
    As = [advection_1d(p, N, periodic, cd) for N, cd in zip(Ns, c)]
    T = kron3(As[0], Ms[1], Ms[2]) + kron3(Ms[0], As[1], Ms[2]) + kron3(Ms[0], Ms[1], As[2])
    return to_dof_order(T, p, Ns)


def cartesian_dof_points(p, Ns):
    """Physical dof coordinates of the identity-mapped mesh, oracle order."""
    k = p + 1
    x = gl_nodes(k)
    Nx, Ny, Nz = Ns
    pts = np.zeros((Nx * Ny * Nz * k ** 3, 3))
    for iz in range(Nz):
        for iy in range(Ny):
            for ix in range(Nx):
                c = ix + Nx * (iy + Ny * iz)
                for i2 in range(k):
                    for i1 in range(k):
                        for i0 in range(k):
                            pts[c * k ** 3 + i0 + k * (i1 + k * i2)] = (
                                (ix + x[i0]) / Nx, (iy + x[i1]) / Ny, (iz + x[i2]) / Nz)
    return pts
