"""Implicit (backward Euler) time step solved by Newton-Krylov iterations on
the GPU, the matrix-free use of the JVP (the paper integrates explicitly,
Sec. 2.1; the RHS Jacobian is its Eq. "jacobian_rhs").

One step solves F(X) = X - U - dt R(X) = 0: Newton updates X <- X + d with
(I - dt J(X)) d = -F(X), each linear system solved by restarted GMRES whose
matrix-vector product is X -> V - dt sdrt_jvp(X, V).  All vectors are device
arrays in the mesh's state layout (padding entries stay zero)."""


def gmres(matvec, b, x0=None, tol=1e-10, restart=30, maxiter=300):
    """Restarted GMRES.  The Arnoldi basis is a device matrix; each new vector
    is orthogonalised by classical Gram-Schmidt with one re-orthogonalisation
    (two pairs of matrix-vector products on the device), and only the new
    Hessenberg column (k + 2 numbers) comes to the host, once per iteration,
    for the Givens rotations and the convergence test.  Returns (x, iterations,
    relative residual)."""
    import numpy as np
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
        Q = torch.empty((m + 1, b.numel()), dtype=b.dtype, device=b.device)
        Q[0] = r.reshape(-1) / beta
        H = np.zeros((m + 1, m))
        cs, sn, g = np.zeros(m), np.zeros(m), np.zeros(m + 1)
        g[0] = beta
        k_used = 0
        for k in range(m):
            w = matvec(Q[k].reshape(b.shape)).reshape(-1)
            Qk = Q[:k + 1]
            h = Qk @ w
            w = w - Qk.T @ h
            h2 = Qk @ w                                          # re-orthogonalisation
            w = w - Qk.T @ h2
            nrm = torch.linalg.vector_norm(w)
            col = torch.cat([h + h2, nrm[None]]).cpu().numpy()   # the one transfer of the iteration
            H[:k + 2, k] = col
            if col[k + 1] > 0:
                Q[k + 1] = w / nrm
            for i in range(k):                                   # previous rotations
                t = cs[i] * H[i, k] + sn[i] * H[i + 1, k]
                H[i + 1, k] = -sn[i] * H[i, k] + cs[i] * H[i + 1, k]
                H[i, k] = t
            den = np.hypot(H[k, k], H[k + 1, k])
            cs[k], sn[k] = H[k, k] / den, H[k + 1, k] / den
            H[k, k] = den
            H[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = cs[k] * g[k]
            k_used = k + 1
            it += 1
            if abs(g[k + 1]) / bnorm <= tol or col[k + 1] <= 0:
                break
        y = np.linalg.solve(np.triu(H[:k_used, :k_used]), g[:k_used])
        x = x + (Q[:k_used].T @ torch.from_numpy(y).to(Q.device, Q.dtype)).reshape(b.shape)
        rel = abs(g[k_used]) / bnorm
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
