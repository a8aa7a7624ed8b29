"""FP64 oracle of the travel-time tomography forward model and its gradient.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper's first example (Sec. 4.1) predicts station-to-station group
travel times with the fast marching method of Rawlinson & Sambridge (2004)
and computes the derivatives of the misfit by tracing ray paths through the
computed travel-time field (Sec. 3; Sec. 4.1, about 0.08 forward costs).
The likelihood is the Gaussian of Eq. (26) with one standard deviation per
travel time. The paper fixes neither the order of the scheme nor how rays are
traced, so this oracle takes these readings:

  * velocity lives on the nodes of a regular ny x nx grid of spacing h (km);
    stations sit on nodes;
  * travel times solve the first-order upwind (Godunov) discretisation of
    the eikonal equation |grad T| = 1 / v, computed by fast marching:
    nodes are accepted in increasing time from a heap, and a node's trial
    time uses only accepted neighbours;
  * one fast-marching solve per source station s = 0 .. ns-2; the data are
    the times at the stations r > s, ordered s-major (pair index
    s * ns - s * (s + 1) / 2 + r - s - 1);
  * a ray starts at the receiver node and steps a fixed length ds (in node
    spacings) against the travel-time gradient; the gradient at a point is
    the bilinear interpolation of nodal gradients, which are central
    differences inside the grid and one-sided differences on its edge
    (numpy.gradient with unit spacing); a step that would leave the grid is
    clipped to it; the ray stops when it is within ds of the source (or its
    gradient vanishes, or after max_steps) and ends with a straight segment
    to the source;
  * each segment adds its length times the bilinear weights of its
    midpoint to the four surrounding nodes: the ray's sensitivity to nodal
    slowness, dT/ds_k = h * sum_seg len * w_k; the velocity derivative is
    dT/dv_k = -dT/ds_k / v_k^2.

Distances inside the ray tracer are in node spacings; times in seconds.
"""
import heapq

import numpy as np


def pair_index(s, r, ns):
    """Position of the travel time from station s to station r > s."""
    return s * ns - s * (s + 1) // 2 + (r - s - 1)


def godunov_time(a, b, f):
    """Upwind update of one node: a and b are the smaller neighbour times
    along the two axes (inf if none is known), f = h / v at the node. The
    solution of ((t-a)^+)^2 + ((t-b)^+)^2 = f^2 (Rawlinson & Sambridge 2004,
    first order)."""
    lo, hi = min(a, b), max(a, b)
    if not np.isfinite(lo):
        return np.inf
    if hi - lo >= f:
        return lo + f
    return 0.5 * (lo + hi + np.sqrt(2.0 * f * f - (hi - lo) ** 2))


def _known_min(T, known, nodes):
    vals = [T[p] for p in nodes if known[p]]
    return min(vals) if vals else np.inf


def fast_marching(v, h, src):
    """Travel times T[ny][nx] (s) from the node src = (i, j) through the
    nodal velocity map v (km/s) with spacing h (km)."""
    v = np.asarray(v, dtype=np.float64)
    ny, nx = v.shape
    f = h / v
    T = np.full((ny, nx), np.inf)
    known = np.zeros((ny, nx), dtype=bool)
    T[src] = 0.0
    heap = [(0.0, src)]
    while heap:
        t, (i, j) = heapq.heappop(heap)
        if known[i, j]:
            continue                      # a stale heap entry
        known[i, j] = True
        for k, l in ((i - 1, j), (i + 1, j), (i, j - 1), (i, j + 1)):
            if not (0 <= k < ny and 0 <= l < nx) or known[k, l]:
                continue
            a = _known_min(T, known, [(k, m) for m in (l - 1, l + 1) if 0 <= m < nx])
            b = _known_min(T, known, [(m, l) for m in (k - 1, k + 1) if 0 <= m < ny])
            tn = godunov_time(a, b, f[k, l])
            if tn < T[k, l]:
                T[k, l] = tn
                heapq.heappush(heap, (tn, (k, l)))
    return T


def _bilinear_cell(y, x, ny, nx):
    i0 = min(int(np.floor(y)), ny - 2)
    j0 = min(int(np.floor(x)), nx - 2)
    return i0, j0, y - i0, x - j0


def _bilinear(F, y, x):
    ny, nx = F.shape
    i0, j0, fy, fx = _bilinear_cell(y, x, ny, nx)
    return ((1 - fy) * ((1 - fx) * F[i0, j0] + fx * F[i0, j0 + 1])
            + fy * ((1 - fx) * F[i0 + 1, j0] + fx * F[i0 + 1, j0 + 1]))


def default_max_steps(ny, nx, ds):
    return int(4 * (ny + nx) / ds)


def trace_ray(T, src, rcv, ds=0.5, max_steps=None):
    """Ray from the receiver node rcv back to the source node src through
    the travel-time field T (steepest descent, fixed step ds in node
    spacings). Returns the list of segments ((y0, x0), (y1, x1))."""
    ny, nx = T.shape
    if max_steps is None:
        max_steps = default_max_steps(ny, nx, ds)
    gy, gx = np.gradient(T)
    s = np.array(src, dtype=np.float64)
    p = np.array(rcv, dtype=np.float64)
    segs = []
    for _ in range(max_steps):
        if np.hypot(*(p - s)) <= ds:
            break
        g = np.array([_bilinear(gy, *p), _bilinear(gx, *p)])
        n = np.hypot(*g)
        if n == 0.0:
            break
        q = p - ds * g / n
        q[0] = min(max(q[0], 0.0), ny - 1.0)
        q[1] = min(max(q[1], 0.0), nx - 1.0)
        segs.append((p.copy(), q.copy()))
        p = q
    segs.append((p.copy(), s.copy()))
    return segs


def ray_sensitivity(segs, ny, nx):
    """sum over segments of length * bilinear weights of the midpoint,
    [ny][nx], in node spacings (the ray's slowness kernel divided by h)."""
    K = np.zeros((ny, nx))
    for p, q in segs:
        L = np.hypot(*(q - p))
        m = 0.5 * (p + q)
        i0, j0, fy, fx = _bilinear_cell(m[0], m[1], ny, nx)
        K[i0, j0] += L * (1 - fy) * (1 - fx)
        K[i0, j0 + 1] += L * (1 - fy) * fx
        K[i0 + 1, j0] += L * fy * (1 - fx)
        K[i0 + 1, j0 + 1] += L * fy * fx
    return K


def _node(k, nx):
    return (int(k) // nx, int(k) % nx)


def traveltimes(v, h, stations):
    """Predicted travel times [ns (ns-1) / 2] for one velocity map v[ny][nx]."""
    v = np.asarray(v, dtype=np.float64)
    ny, nx = v.shape
    ns = len(stations)
    out = np.empty(ns * (ns - 1) // 2)
    for s in range(ns - 1):
        T = fast_marching(v, h, _node(stations[s], nx))
        for r in range(s + 1, ns):
            out[pair_index(s, r, ns)] = T[_node(stations[r], nx)]
    return out


def misfit_gradient(v, h, stations, dobs, sigma, ds=0.5, sources=None):
    """Misfit J = sum_i (d_i(v) - d_i^obs)^2 / (2 sigma_i^2) (Eq. 26) and
    dJ/dv [ny][nx] from ray sensitivities, for one velocity map. sources
    restricts the sum to the pairs whose source station is listed."""
    v = np.asarray(v, dtype=np.float64)
    ny, nx = v.shape
    ns = len(stations)
    J = 0.0
    Ksum = np.zeros((ny, nx))
    for s in (range(ns - 1) if sources is None else sources):
        T = fast_marching(v, h, _node(stations[s], nx))
        for r in range(s + 1, ns):
            i = pair_index(s, r, ns)
            res = T[_node(stations[r], nx)] - dobs[i]
            J += 0.5 * res * res / (sigma[i] * sigma[i])
            segs = trace_ray(T, _node(stations[s], nx), _node(stations[r], nx), ds)
            Ksum += (res / (sigma[i] * sigma[i])) * ray_sensitivity(segs, ny, nx)
    grad = -h * Ksum / (v * v)
    return J, grad


def traveltimes_batch(V, h, stations, ny, nx):
    return np.stack([traveltimes(np.asarray(x).reshape(ny, nx), h, stations)
                     for x in V])


def misfit_gradient_batch(V, h, stations, dobs, sigma, ny, nx, ds=0.5):
    Js, Gs = [], []
    for x in V:
        J, g = misfit_gradient(np.asarray(x).reshape(ny, nx), h, stations,
                               dobs, sigma, ds)
        Js.append(J)
        Gs.append(g.reshape(-1))
    return np.array(Js), np.stack(Gs)
