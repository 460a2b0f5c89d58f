"""Implicit (backward Euler) time step solved by Newton-Krylov iterations on
the GPU, the matrix-free use of the JVP (the paper integrates explicitly,
Sec. 2.1; the RHS Jacobian is its Eq. "jacobian_rhs").

One step solves F(X) = X - U - dt R(X) = 0: Newton updates X <- X + d with
(I - dt J(X)) d = -F(X), each linear system solved by restarted GMRES whose
matrix-vector product is X -> V - dt sdrt_jvp(X, V).  All vectors are device
arrays in the mesh's state layout (padding entries stay zero)."""


def gmres(matvec, b, x0=None, tol=1e-10, restart=30, maxiter=300):
    """Restarted GMRES (modified Gram-Schmidt Arnoldi, Givens rotations).
    Returns (x, iterations, relative residual)."""
    import torch
    x = torch.zeros_like(b) if x0 is None else x0.clone()
    bnorm = float(torch.linalg.vector_norm(b))
    if bnorm == 0.0:
        return x, 0, 0.0
    it = 0
    rel = 1.0
    while it < maxiter:
        r = b - matvec(x)
        beta = float(torch.linalg.vector_norm(r))
        rel = beta / bnorm
        if rel <= tol:
            break
        m = min(restart, maxiter - it)
        Q = [r / beta]
        H = torch.zeros(m + 1, m, dtype=torch.float64)
        cs = torch.zeros(m, dtype=torch.float64)
        sn = torch.zeros(m, dtype=torch.float64)
        g = torch.zeros(m + 1, dtype=torch.float64)
        g[0] = beta
        k_used = 0
        for k in range(m):
            w = matvec(Q[k])
            for i in range(k + 1):
                H[i, k] = float(torch.dot(Q[i], w))
                w = w - H[i, k] * Q[i]
            H[k + 1, k] = float(torch.linalg.vector_norm(w))
            if H[k + 1, k] > 0:
                Q.append(w / H[k + 1, k])
            for i in range(k):                                   # previous rotations
                t = cs[i] * H[i, k] + sn[i] * H[i + 1, k]
                H[i + 1, k] = -sn[i] * H[i, k] + cs[i] * H[i + 1, k]
                H[i, k] = t
            den = (H[k, k] ** 2 + H[k + 1, k] ** 2).sqrt()
            cs[k], sn[k] = H[k, k] / den, H[k + 1, k] / den
            H[k, k] = den
            H[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = cs[k] * g[k]
            k_used = k + 1
            it += 1
            if abs(float(g[k + 1])) / bnorm <= tol or len(Q) <= k + 1:
                break
        y = torch.linalg.solve_triangular(H[:k_used, :k_used], g[:k_used, None], upper=True)[:, 0]
        for i in range(k_used):
            x = x + float(y[i]) * Q[i]
        rel = abs(float(g[k_used])) / bnorm
        if rel <= tol:
            break
    return x, it, rel


def backward_euler_step(mesh, U, dt, newton_tol=1e-10, max_newton=20, gmres_tol=1e-10, restart=30):
    """X solving X - U - dt R(X) = 0 (FP64 meshes).  Returns (X, info) with the
    Newton history of ||F|| / ||U|| and the GMRES iterations per Newton step."""
    import torch
    if U.dtype != torch.float64:
        raise ValueError("the Newton-Krylov step runs in FP64")
    R = torch.zeros_like(U)
    JV = torch.zeros_like(U)
    X = U.clone()
    unorm = float(torch.linalg.vector_norm(U))
    hist, gits = [], []
    for _ in range(max_newton):
        mesh.residual(X, R)
        F = X - U - dt * R
        fn = float(torch.linalg.vector_norm(F)) / unorm
        hist.append(fn)
        if fn <= newton_tol:
            break

        def matvec(v):
            mesh.jvp(X, v, JV)
            return v - dt * JV

        d, it, _ = gmres(matvec, -F, tol=gmres_tol, restart=restart)
        gits.append(it)
        X = X + d
    mesh.sync()
    return X, {"residual_history": hist, "gmres_iterations": gits}
