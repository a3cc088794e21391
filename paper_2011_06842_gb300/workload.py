"""Algorithmic work of one PCG iteration: the paper's FLOP model and the byte
count used for the roofline.

``pcg_flops_per_iter`` is the per-iteration formula of Table FEWHAFLOPs
(Sec. 7.1), generalised to layers of different sizes by summing the
per-layer terms.  ``aug_init_flops`` and ``aug_proj_flops`` are the two
augmented rows of that table (per iteration / per solve, n_augIter factor
left to the caller).

``bytes_per_iter`` counts the algorithmic traffic of one iteration of the
persistent solver: every intermediate written once and read once, solver
vectors at their storage width.
"""


def pcg_flops_per_iter(G_NGS, G_LGS, n_s, layer_sizes):
    G = G_NGS + G_LGS
    L = len(layer_sizes)
    f = (14 * G_LGS + 2 * G_NGS + 12 * G) * n_s ** 2 + 4 * G * n_s
    f += ((L - 1) * (15.6 * G_LGS + 18 * G_NGS) + L * (G - 1)) * (n_s + 1) ** 2
    f += sum(176.0 / 3.0 * (4 * n * n - 1) + 13 * n * n for n in layer_sizes)
    return f


def aug_init_flops(layer_sizes):
    return 9 * sum(n * n for n in layer_sizes)


def aug_proj_flops(layer_sizes):
    return 4 * sum(n * n for n in layer_sizes)


def aug_memory_bytes(layer_sizes, k, word=4):
    """(2 n_lay^2 L + 1) k words of extra storage (Sec. 7.2)."""
    return (2 * sum(n * n for n in layer_sizes) + 1) * k * word


def geometry_counts(geom):
    g_lgs = sum(1 for g in geom.gs if g.H > 0)
    return dict(G_NGS=len(geom.gs) - g_lgs, G_LGS=g_lgs, n_s=geom.n_sub,
                layer_sizes=[l.n for l in geom.layers])


def bytes_per_iter(geom, word=4, augmented=True):
    """Algorithmic bytes of one solver iteration (operator + vector updates).

    Operator intermediates, each written once and read once: nodal layers (n),
    adjoint wavefronts (G (n_s+1)^2).  Solver vectors: read p, r, c, q, J^{-1},
    prior, p_m, q_m (augmented) and write p, q, c, r (q and p land in the
    recycled-basis slot, no copy).
    """
    n = sum(l.n * l.n for l in geom.layers)
    G = len(geom.gs)
    m2 = (geom.n_sub + 1) ** 2
    op = 2 * n + 2 * G * m2
    vec_reads = 6 + (2 if augmented else 0)
    vec_writes = 4
    return word * (op + (vec_reads + vec_writes) * n)


def solve_bytes(geom, iters, kv, word=4):
    """Algorithmic bytes of one time step of the solver: right-hand side and
    warm restart, projection onto kv recycled directions, and iters iterations.

    RHS: slopes read, adjoint wavefronts written and read, b_prev read and
    written, r read and written.  Projection: the Gram matrix and P^T r read
    2 kv + 1 vectors; the update reads c, r, kv p and kv q and writes c, r;
    the dots after it read r and kv q.
    """
    n = sum(l.n * l.n for l in geom.layers)
    G = len(geom.gs)
    m2 = (geom.n_sub + 1) ** 2
    rhs = 2 * geom.n_sub ** 2 * G + 2 * G * m2 + 4 * n
    init = (5 * kv + 6) * n if kv > 0 else 0
    return word * (rhs + init) + iters * bytes_per_iter(geom, word, augmented=kv > 0)


def op_intermediate_words(geom):
    """Operator intermediates of one application of M, each written once and
    read once: nodal layers (n), forward wavefronts (G (n_s+1)^2), slopes
    (G 2 n_s^2), adjoint wavefronts (G (n_s+1)^2), adjoint layers (n)."""
    n = sum(l.n * l.n for l in geom.layers)
    G = len(geom.gs)
    m2 = (geom.n_sub + 1) ** 2
    return 2 * (2 * n + 2 * G * m2 + 2 * G * geom.n_sub ** 2)


def reference_bytes_per_iter(geom, word=4):
    """The per-iteration count of the scope table's measurement row: solver
    vectors ~14 n words (read p, J^{-1}, p_m, q_m, c, r, q, z; write q, c, r,
    z, p, the basis copy) plus the operator intermediates
    (op_intermediate_words), written once and read once, whether or not an
    implementation keeps them in registers or shared memory (the fused WFS
    phase never stores the slopes)."""
    n = sum(l.n * l.n for l in geom.layers)
    return word * (14 * n + op_intermediate_words(geom))


def reference_solve_bytes(geom, iters, k, word=4, augmented=True):
    """Bytes of one time step under the same count: iters iterations, the
    right-hand side and initial projection (~1.5 operator-equivalents for
    augmented PCG, the right-hand side alone, 0.5, for plain PCG) and the
    9 n k projection reads of the recycled basis (augmented only; the FLOP
    table's 9 n_lay^2 L augmented term)."""
    n = sum(l.n * l.n for l in geom.layers)
    op = op_intermediate_words(geom)
    extra = (1.5 * op + 9 * n * k) if augmented else 0.5 * op
    return iters * reference_bytes_per_iter(geom, word) + word * extra
