"""Fill orders for the oracle, written from their definitions.

Test infrastructure only.  Each function returns a list of (i, j) cells.  The
orders always start with row 0 (its cells are then fixed by a prefix, e.g.
the identity row of Section 2.2).

For vertically symmetric squares only left-half cells (j < N/2) are listed:
the right half follows from A[i][N-1-j] = N-1-A[i][j] (Section 5.4).
"""


def _cols(n, vsym):
    return range(n // 2) if vsym else range(n)


def row0(n, vsym=False):
    return [(0, j) for j in _cols(n, vsym)]


def md_ad_rows(n, vsym=False, first_rows=1):
    """Rows 0..first_rows-1, then the main diagonal top to bottom, then the
    anti-diagonal top to bottom, then the remaining cells row by row, left to
    right (cells already listed are skipped).  With ``vsym`` only left-half
    cells are used, so the main diagonal contributes rows i < N/2 and the
    anti-diagonal rows i >= N/2."""
    seen = set()
    out = []

    def add(c):
        if c not in seen and c[1] in _cols(n, vsym):
            seen.add(c)
            out.append(c)

    for i in range(first_rows):
        for j in _cols(n, vsym):
            add((i, j))
    for i in range(n):
        add((i, i))
    for i in range(n):
        add((i, n - 1 - i))
    for i in range(n):
        for j in _cols(n, vsym):
            add((i, j))
    return out


def row_major(n, vsym=False):
    return [(i, j) for i in range(n) for j in _cols(n, vsym)]


def hourglass(n):
    """Row 0, main diagonal, anti-diagonal, last row (the cells of an
    hourglass design, Section 4.2), then rows 1..N-2."""
    seen = set()
    out = []

    def add(c):
        if c not in seen:
            seen.add(c)
            out.append(c)

    for j in range(n):
        add((0, j))
    for i in range(n):
        add((i, i))
    for i in range(n):
        add((i, n - 1 - i))
    for j in range(n):
        add((n - 1, j))
    for i in range(n):
        for j in range(n):
            add((i, j))
    return out


def hourglass_cells(n, vsym=False):
    """The cells of an hourglass design (Section 4.2) in the order they are
    filled: row 0, main diagonal, anti-diagonal, last row (left half only
    with vsym, where a diagonal cell's mirror lies on the other diagonal)."""
    w = n // 2 if vsym else n
    seen = set()
    out = []

    def add(c):
        if c not in seen and c[1] < w:
            seen.add(c)
            out.append(c)

    for j in range(n):
        add((0, j))
    for i in range(n):
        add((i, i))
    for i in range(n):
        add((i, n - 1 - i))
    for j in range(n):
        add((n - 1, j))
    return out


def identity(n, vsym=False):
    """Values of row 0 fixed to 0..N-1 (left half only when vsym)."""
    return [j for j in _cols(n, vsym)]


def heuristic_complete(n, kept, diagonal=True, vsym=False, squares=False):
    """Section 2.3: starting from the `kept` cells (row 0 for a whole
    order), repeatedly take the unassigned cell with the largest
    V = r_i + c_j + md(i,j) + ad(i,j) -- the numbers of assigned cells in its
    row, its column and, when it lies on them, the two diagonals -- ties
    going to the first cell in row-major order.  When an assignment leaves
    one unassigned cell in one of its lines (row, column, main diagonal,
    anti-diagonal, looked at in that order), that cell is taken next
    (first-in first-out).  With vsym only left-half cells exist: a row has
    N//2 of them, a column N, and the diagonals form one line made of the
    left cells on either diagonal.  squares=True: V is the sum of the squares
    of those numbers instead (a variant the paper does not have).  Returns
    kept + the appended cells."""
    w = n // 2 if vsym else n
    lines = [[(i, j) for j in range(w)] for i in range(n)]
    lines += [[(i, j) for i in range(n)] for j in range(w)]
    if diagonal and not vsym:
        lines.append([(i, i) for i in range(n)])
        lines.append([(i, n - 1 - i) for i in range(n)])
    elif diagonal and vsym:
        # left cells of the main diagonal (upper rows) and of the
        # anti-diagonal (lower rows); an odd order's centre is not a left cell
        lines.append([(i, i) for i in range(w)] + [(i, n - 1 - i) for i in range(n - w, n)])
    of_cell = {}
    for li, line in enumerate(lines):
        for c in line:
            of_cell.setdefault(c, []).append(li)
    assigned = set()
    out = []
    queue = []

    def assign(c, forced_rule):
        assigned.add(c)
        out.append(c)
        if not forced_rule:
            return
        for li in of_cell[c]:
            rest = [x for x in lines[li] if x not in assigned]
            if len(rest) == 1:
                queue.append(rest[0])

    for c in kept:
        assign(tuple(c), False)
    while len(out) < n * w:
        cell = None
        while queue:
            x = queue.pop(0)
            if x not in assigned:
                cell = x
                break
        if cell is None:
            best = -1
            for i in range(n):
                for j in range(w):
                    if (i, j) in assigned:
                        continue
                    counts = [sum(1 for x in lines[li] if x in assigned) for li in of_cell[(i, j)]]
                    v = sum(c * c for c in counts) if squares else sum(counts)
                    if v > best:
                        best, cell = v, (i, j)
        assign(cell, True)
    return out


def trim_tail(n, order, keep, window=6, diagonal=True, vsym=False):
    """The order shortened so that every count stays the same.

    Why a final run may go: say the last k cells of a full order all lie in
    row r, none on a diagonal.  Fill every other cell validly.  Then each of
    the k cells is the only empty cell of its column, so its value is the
    one value that column lacks (Section 2.4.1 computes such a last value
    directly).  Take a value v.  The n-1 other rows are full, so v fills n-1
    cells there, plus one in row r unless row r lacks v; the n-k columns
    without an empty cell hold v once each; so the k columns of the run hold
    v (n-1) + [r has v] - (n-k) times, and (k-1) + [r has v] of them have it:
    exactly one of them lacks v when row r lacks v, none when it has it.
    The forced values are therefore the k values row r lacks, each once, and
    no diagonal constrains those cells: the filling completes in exactly one
    way.  A count over the first len-k cells (which counts fillings of
    them) equals the count over the whole order.  Columns instead of rows:
    the same with the roles swapped.

    The rule: take the cells of the last cell's row among the last `window`
    cells (none of the first `keep`), move them to the end keeping their
    order, and count the run at the end that lies on that row and on neither
    diagonal; the same with the last cell's column; keep the line with the
    longer run (the row on a tie, nothing if both are empty) and drop its
    run, leaving at least one cell after the first `keep`.  Only for an
    order that lists every cell (every left-half cell with vertical
    symmetry); anything else is returned as it is.

    Vertical symmetry (Section 5.4: the order lists the left half, the right
    half is A[i][N-1-j] = N-1-A[i][j]): a row is valid when its left half
    holds one value of each pair {v, N-1-v}, a column when it holds every
    value.  A row's run still consists of columns' last open cells.  Take a
    pair P: the N-1 full rows hold one P value each in their left halves,
    the N/2 left columns two each (both values), so the left half lacks
    N - (N-1) - a = 1 - a of them, where a (0 or 1) is the number of P
    values the run's row already holds -- all in the run's columns, at most
    one per column.  So the run's row receives one value of each pair it
    lacks and none of a pair it has: valid, and again unique.  A column's
    run does not work here: a row's last left cell may take either value of
    its missing pair, so it is not forced."""
    order = [tuple(map(int, c)) for c in order]
    w = n // 2 if vsym else n
    if (vsym and n % 2) or len(order) != n * w or len(order) <= keep + 1:
        return order
    start = max(keep, len(order) - window)
    best, best_k = order, 0
    for axis in ((0,) if vsym else (0, 1)):
        line = order[-1][axis]
        on = [c for c in order[start:] if c[axis] == line]
        off = [c for c in order[start:] if c[axis] != line]
        cand = order[:start] + off + on
        k = 0
        for c in reversed(cand):
            if c[axis] != line or k == len(order) - keep - 1:
                break
            if diagonal and (c[0] == c[1] or c[0] + c[1] == n - 1):
                break
            k += 1
        if k > best_k:
            best, best_k = cand, k
    return best[:len(best) - best_k]
