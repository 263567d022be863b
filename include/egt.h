/*
 * egt.h -- C-ABI of the B300 Excessive Gap Technique library (libegt.so).
 *
 * Solves the sequence-form bilinear saddle point of a two-player zero-sum
 * poker river endgame,  min_{x in X} max_{y in Y} <x, A y>  (Eq. 1 / Eq. 2),
 * with EGT and the dilated entropy distance (Sec. 3, Sec. 5, Algorithms 1-4).
 * x is player 1 (moves first, minimises), y is player 2 (maximises); A holds
 * the expected payoff to player 2, chance-normalised per hand dealt.
 *
 * Conventions shared by every call
 * --------------------------------
 * - Every function returns an egt_status and never aborts; on failure a
 *   thread-local message is available from egt_last_error().
 * - The caller owns every pointer it passes; the library never frees caller
 *   memory.  An egt_game owns its device tables and solver state and frees
 *   them in egt_destroy_game.
 * - "device" pointers are CUDA global memory on the game's device; "host"
 *   pointers are ordinary CPU memory.
 * - Strategy and gradient vectors are laid out [seq][hand] with a leading
 *   dimension ld (egt_dims.ld, a multiple of 32 >= H, at most 1536): element (s, h) is at
 *   s * ld + h.  Hands are in ascending strength order (ties by input index),
 *   see egt_hand_order.  Columns h >= H are ignored on input and written as
 *   0 on output.  Vector base pointers must be 16-byte aligned.
 * - stream: a cudaStream_t (NULL = legacy default stream).  Kernels run on it;
 *   calls that return host values synchronise it.  Calls on one game share
 *   its scratch memory: issue them on one stream (or otherwise serialise).
 *
 * Game model (Sec. 7, subgame description) and the betting reading used here
 * --------------------------------------------------------------------------
 * Chance deals each player a private hand from that player's range (hands
 * sharing a card are never dealt together); player 1 acts first; fold ends
 * the game, call or two opening checks go to showdown (stronger hand wins the
 * stake, ties pay 0).  Each player has pot/2 in; the loser pays pot/2 plus
 * their river chips.  Not facing a bet: check, or bet f * pot_total for each
 * menu fraction f.  Facing a bet: fold, call, or raise by call + f *
 * (pot_total + call).  Sizes that reach the remaining stack are dropped;
 * all-in is offered (if enabled) while the number of bets is below raise_cap
 * and chips remain after calling; raise_cap counts the opening bet and the
 * raises; there is no fold when not facing a bet.
 *
 * Canonical numbering: the public tree is walked depth first with actions in
 * the order fold, check/call, menu sizes, all-in; a player's information sets
 * (simplexes) are sorted by (level b_Q^j, preorder index of the public node);
 * sequences are numbered simplex by simplex in action order; terminals in
 * preorder.  The empty sequence is not stored.
 */
#ifndef EGT_H_
#define EGT_H_

#include <stdint.h>

#if defined(__GNUC__)
#define EGT_API __attribute__((visibility("default")))
#else
#define EGT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct egt_game egt_game;

typedef enum {
  EGT_OK = 0,
  EGT_ERR_INVALID_ARG = 1,     /* bad pointer, size, player, range, card id, ... */
  EGT_ERR_OOM = 2,             /* device or host allocation failed */
  EGT_ERR_CUDA = 3,            /* a CUDA runtime call or kernel launch failed */
  EGT_ERR_NUMERIC = 4,         /* a NaN / Inf appeared in a value */
  EGT_ERR_TAU_UNDERFLOW = 5,   /* Alg. 4 halved tau below 2^-30 */
  EGT_ERR_NOT_CONVERGED = 6,   /* egt_solve hit max_iters above its gap target */
  EGT_ERR_TIMEOUT = 7          /* reserved: a bounded device wait gave up */
} egt_status;

/* One river endgame (all pointers host, read during egt_create_game only).
 * hand_cards: [n_hands][hand_size] card ids in [0, n_cards), distinct within a
 *   hand, no two hands equal; hand_size is 1 or 2.
 * strength: [n_hands], higher wins, equal = tie.
 * range[p]: [n_hands] >= 0 finite, not all zero; normalised internally.
 * pot, stack: chips (stack = remaining chips of each player, equal stacks).
 * bb: chips per big blind; gaps are reported in mbb = bb / 1000 per hand.
 * bet_fracs: [n_bets] pot fractions > 0 in menu order.
 * menus: NULL = the one menu (bet_fracs, allin) for every decision, no fold
 *   unless facing a bet.  Else [2][4] menus, menus[p][k] for player p after k
 *   bets or raises in the river so far (k = 3 for three or more): the pot
 *   fractions of its bets / raises, whether all-in is offered and whether fold
 *   is offered when not facing a bet (Sec. 7's Libratus abstraction gives
 *   each player its own sizes for the opening, facing the first bet, facing a
 *   raise and facing later raises).  raise_cap still bounds the bets. */
typedef struct {
  int32_t n;              /* sizes */
  const double* fracs;    /* [n] pot fractions > 0 in menu order */
  int32_t allin;          /* all-in offered */
  int32_t fold;           /* fold offered when not facing a bet */
} egt_menu;

typedef struct {
  int32_t n_cards;
  int32_t hand_size;
  int32_t n_hands;
  const int32_t* hand_cards;
  const int32_t* strength;
  const double* range[2];
  double pot;
  double stack;
  double bb;
  int32_t n_bets;
  const double* bet_fracs;
  int32_t allin;
  int32_t raise_cap;
  const egt_menu* menus;  /* NULL or [2][4], see above */
} egt_game_desc;

/* Sizes and constants of a compiled game.
 * S[p] sequences, J[p] simplexes (information sets per hand), L[p] levels of
 * player p's per-hand treeplex; T terminals (n_fold of them folds); H hands;
 * ld leading dimension; Z chance normaliser (sum over compatible hand pairs
 * of r1 r2); normA = max |A_ij| (the l1 operator norm, Sec. 3); M[p] = max l1
 * norm of player p's strategy space (DGF modulus 1/M, Sec. 5); Omega[p] = max
 * minus min of the dilated entropy over it (Sec. 3). */
typedef struct {
  int32_t H, ld;
  int32_t S[2], J[2], L[2];
  int32_t T, n_fold;
  double Z, normA, M[2], Omega[2];
  int64_t table_bytes;   /* bytes of compiled tables uploaded by egt_create_game */
  int64_t device_bytes;  /* device memory the game holds (tables and solver state); also
                            filled for host-only games, so a caller can size admission */
} egt_dims;

/* Compile the game (betting tree, treeplex tables, hand/card tables) and
 * upload it to `device`; allocates the game's device memory (tables, solver
 * state, scratch).  *out receives the handle.  device = -1 compiles the host
 * tables only: the query calls work, every compute call returns INVALID_ARG,
 * and no CUDA call is made.  Errors: INVALID_ARG on an invalid description,
 * OOM, CUDA. */
EGT_API egt_status egt_create_game(const egt_game_desc* desc, int32_t device, void* stream, egt_game** out);

/* Free everything the game owns (synchronises its device).  NULL is a no-op. */
EGT_API egt_status egt_destroy_game(egt_game* game);

EGT_API egt_status egt_dims_query(const egt_game* game, egt_dims* out);

/* order[k] (host, [H]) = input index of the hand at sorted position k. */
EGT_API egt_status egt_hand_order(const egt_game* game, int32_t* order);

/* Per-hand treeplex of player p (Sec. 4 notation), host arrays of length J[p]:
 * parent sequence p_j (-1: q_{p_j} = 1), first sequence of I_j, n_j, level
 * b_Q^j, and the DGF weight beta_j = 2 + sum over child simplexes 2 beta_k
 * (Sec. 5).  Any pointer may be NULL. */
EGT_API egt_status egt_treeplex_query(const egt_game* game, int32_t player, int32_t* parent,
                              int32_t* first_seq, int32_t* n_actions, int32_t* level,
                              double* beta);

/* Terminals in preorder, host arrays of length T: sigma_1(b), sigma_2(b),
 * kind (0 fold, 1 showdown), coef (fold: payoff to player 2; showdown: stake
 * paid by the weaker hand).  Any pointer may be NULL. */
EGT_API egt_status egt_terminal_query(const egt_game* game, int32_t* seq1, int32_t* seq2,
                              int32_t* kind, double* coef);

/* Gradient product (Sec. 3: grad f = A y, grad phi = A^T x).
 * player 0: out[S0][ld] = A in, in = y [S1][ld];
 * player 1: out[S1][ld] = A^T in, in = x [S0][ld].  Device pointers, in != out.
 * Computed per terminal with card-removal inclusion-exclusion (folds) and
 * strength-sorted prefix sums with per-card corrections (showdowns).  Each
 * term w = r x in enters its column's sums as one int64 at a power-of-two
 * scale (within 2^-47 |w| + 2^-50 of the column's largest |w|), and the
 * integer sums are exact and rounded once: the output is the FP32 value of
 * r_me / Z x the sum of the sequence's terminal contributions. */
EGT_API egt_status egt_grad(egt_game* game, int32_t player, const float* in, float* out, void* stream);

/* Same product with FP64 input and output (the stopping gap's precision). */
EGT_API egt_status egt_grad_f64(egt_game* game, int32_t player, const double* in, double* out,
                        void* stream);

/* Smoothed best response with the dilated entropy DGF (Sec. 5).
 * player 0: q = argmin_{x in X} <x, g> + mu d_X(x), value = that minimum
 *           (phi_mu(y) when g = A y);
 * player 1: q = argmax_{y in Y} <y, g> - mu d_Y(y), value = that maximum
 *           (f_mu(x) when g = A^T x).
 * g, q_out: device [S_p][ld] (q_out may be NULL to get the value only).
 * value_out: host, may be NULL (then no synchronisation).  mu > 0. */
EGT_API egt_status egt_smoothed_br(egt_game* game, int32_t player, const float* g, double mu,
                           float* q_out, double* value_out, void* stream);

/* Plain best-response value in FP64 (the mu -> 0 limit; Sec. 3 residual):
 * player 0: min_x <x, g>; player 1: max_y <y, g>.  g device [S_p][ld] FP64,
 * value_out host. */
EGT_API egt_status egt_best_response_f64(egt_game* game, int32_t player, const double* g,
                                 double* value_out, void* stream);

/* Saddle-point residual eps_sad(x, y) = max_y' x^T A y' - min_x' x'^T A y (Sec. 3),
 * products and best responses in FP64, in mbb per hand (host out).  x, y device. */
EGT_API egt_status egt_gap(egt_game* game, const float* x, const float* y, double* gap_mbb,
                   void* stream);

/* The same residual as egt_gap, for callers that must not allocate device
 * memory on their path (a serving process whose device memory is reserved up
 * front by another allocator, or a latency-critical loop that cannot take the
 * device-wide synchronisation of cudaMalloc / cudaFree).  The paper has no
 * counterpart: this is a deployment variant.  It allocates nothing: its FP64
 * product vectors and reduction scratch live in one static device array of
 * 2 MiB that every GPU loading the library holds until exit, so games needing
 * more (2 * T * ld * 8 bytes for T terminals, plus about 9 KB) are rejected with
 * INVALID_ARG and a message giving both sizes.  The first call on each device
 * does a one-time set-up, looking up the array's address with that device
 * current; make that first call before any stream capture.  Every call copies
 * the residual to the host and waits for its stream before returning.  All
 * calls share the array (each clears what must start at zero); calls that
 * overlap on the GPU race, so serialise them (one stream).  The game is only
 * read.  x, y device [S_p][ld]; gap_mbb host. */
EGT_API egt_status egt_gap_noalloc(const egt_game* game, const float* x, const float* y,
                                   double* gap_mbb, void* stream);

/* ---- solver (Algorithms 1-4) ---------------------------------------------- */

typedef enum {
  EGT_THEORY = 0,     /* Alg. 1: mu = ||A|| sqrt(M_X M_Y), tau_t = 2/(t+3), alternate by parity */
  EGT_PRACTICAL = 1,  /* "EGT": tuned mu (alpha), tau_t = 2/(t+3), step the player with larger mu */
  EGT_AS = 2          /* "EGT/as": Alg. 3 + 4, aggressive tau with backtracking on EGV < 0 */
} egt_variant;

/* One accepted iteration: t, the player that stepped, back-offs (Alg. 4), its
 * tau, mu after it, EGV (EGT/as; NaN otherwise), the last residual computed
 * before its update (mbb per hand; with gap_every = 1 that of the iterates it
 * started from; NaN if none), and a clock reading at
 * acceptance in ns (the device's global timer for the device engine, the
 * host's steady clock for the host loop): differences within one solve are
 * elapsed time. */
typedef struct {
  int32_t t, player, backoffs;
  double tau, mu[2], egv, gap_mbb;
  uint64_t time_ns;
} egt_iter_log;

/* alpha: practical variants start from mu = alpha ||A|| sqrt(M_X M_Y) and
 *   double both mu while EGV < 0 at the initial point.
 * mu0: if both > 0, the initial mu as given (no guard).
 * eps_mbb: stop once eps_sad <= eps_mbb (checked every gap_every iterations,
 *   FP64); <= 0 runs max_iters.
 * replay: if replay_n > 0, iteration t steps player replay_player[t] with
 *   tau = replay_tau[t] (no EGV check) for replay_n iterations (host arrays).
 * log: optional host array of log_cap entries filled per iteration.
 * engine: EGT_ENGINE_DEVICE (0) runs the iterations in one cooperative launch
 *   (egt_iterate) when the device supports it and no replay is given;
 *   EGT_ENGINE_HOST (1) drives every Step from the host (egt_step).  Both give
 *   the same iterates bit for bit. */
typedef enum { EGT_ENGINE_DEVICE = 0, EGT_ENGINE_HOST = 1 } egt_engine;
typedef struct {
  int32_t variant;
  double alpha;
  double mu0[2];
  double eps_mbb;
  int32_t max_iters;
  int32_t gap_every;
  int32_t replay_n;
  const int32_t* replay_player;
  const double* replay_tau;
  int32_t log_cap;
  egt_iter_log* log;
  int32_t engine;
} egt_solve_opts;

typedef struct {
  int32_t iters, products, backoffs, gap_checks;
  double gap_mbb, mu[2], tau, seconds;
} egt_solve_report;

/* Initial point of Alg. 1 / 3: x_omega = uniform behavioural strategy,
 * y^0 = y_{mu_y}(x_omega), x^0 = x_{mu_x}(y^0) (grad d* with the minus sign
 * restored), mu from opts (variant, alpha, mu0, guard). */
EGT_API egt_status egt_solver_init(egt_game* game, const egt_solve_opts* opts, void* stream);

typedef enum {
  EGT_STEP_PLAIN = 0,   /* one Step (Alg. 2) at tau, always kept */
  EGT_STEP_CHECK = 1,   /* one Step at tau, EGV evaluated, kept iff EGV >= 0 */
  EGT_STEP_DECR = 2     /* Alg. 4: halve tau until EGV >= 0, then keep */
} egt_step_mode;

typedef struct {
  int32_t player, accepted, backoffs, products;
  double tau, egv, mu[2];
} egt_step_info;

/* One Step (Alg. 2) from the solver state; player 0 = x-focused, 1 =
 * y-focused, -1 = the player with the larger mu (tie: y).  *tau_inout is the
 * step size (Decr writes back the accepted one).  info (host) may be NULL. */
EGT_API egt_status egt_step(egt_game* game, int32_t player, double* tau_inout, int32_t mode,
                    egt_step_info* info, void* stream);

/* The intermediate point of the last Step attempt that egt_step ran (Alg. 2,
 * Sec. 3): x_hat = (1 - tau) x + tau x_{mu_x}(y) when x stepped, y_hat
 * likewise when y stepped, in FP32 as the Step used it.  v_hat: device
 * [S_p][ld] of that player (caller-owned); *player (host) receives 0 or 1.
 * A diagnostic for checking each stage of a Step on its own.  INVALID_ARG if
 * no egt_step ran since the last call that reuses the scratch (egt_solver_init,
 * egt_state_set, egt_iterate, egt_solve, a batch step of this game). */
EGT_API egt_status egt_step_point(egt_game* game, float* v_hat, int32_t* player, void* stream);

/* Copy the current iterates (device [S_p][ld], NULL to skip) and mu (host [2]). */
EGT_API egt_status egt_state_get(egt_game* game, float* x, float* y, double* mu, void* stream);

/* Replace the iterates and mu (checkpoint resume); cached products are recomputed. */
EGT_API egt_status egt_state_set(egt_game* game, const float* x, const float* y, const double* mu,
                         void* stream);

/* Checkpoint of a solve: the iterates plus the scalars of the Alg. 1 / 3
 * bookkeeping.  The cached products are not part of it: they are the exact
 * products of the iterates, recomputed on restore. */
typedef struct {
  int32_t t;         /* iterations accepted since egt_solver_init (tau_t = 2 / (t + 3)) */
  double tau;        /* EGT/as step size carried to the next iteration */
  double mu[2];      /* mu_x, mu_y */
  double gap_mbb;    /* last residual in mbb per hand (NaN if none yet) */
} egt_checkpoint;

/* Save: iterates to x, y (device [S_p][ld], either may be NULL) and the scalars
 * to *ck (host).  Restore: a game created from the same description (any
 * device) takes the iterates and scalars, initialised or not; the solve then
 * continues bit for bit as the uninterrupted one (same iterates, mu, tau,
 * residuals).  Restore returns INVALID_ARG for mu <= 0, tau outside (0, 1] or
 * t < 0. */
EGT_API egt_status egt_checkpoint_get(egt_game* game, float* x, float* y, egt_checkpoint* ck, void* stream);
EGT_API egt_status egt_checkpoint_set(egt_game* game, const float* x, const float* y, const egt_checkpoint* ck,
                                      void* stream);

/* eps_sad of the current iterates in mbb per hand (host out), as egt_gap computes
 * it: the stopping test of Alg. 1 / 3. */
EGT_API egt_status egt_state_gap(egt_game* game, double* gap_mbb, void* stream);

/* Continue the solver for up to n_iters iterations of opts->variant on the
 * device: one cooperative launch runs every Step (Alg. 2) with the EGT/as
 * back-off of Alg. 4, the mu / tau bookkeeping and the FP64 residual every
 * opts->gap_every iterations and after the last one, stopping early once it is
 * <= opts->eps_mbb (if > 0).  No host round trip happens inside.  rep (host,
 * may be NULL): iterations run, products, back-offs, residual checks, the last
 * residual (NaN if none yet), mu, tau.  Each grid barrier of the launch waits
 * at most ~2 s; if one runs out the call returns EGT_ERR_TIMEOUT and the
 * solver must be re-initialised.  Replay schedules are not accepted. */
EGT_API egt_status egt_iterate(egt_game* game, const egt_solve_opts* opts, int32_t n_iters,
                               egt_solve_report* rep, void* stream);

/* Run Alg. 1 / practical EGT / Alg. 3 from egt_solver_init to the gap target.
 * x_out, y_out: device, may be NULL.  rep: host, may be NULL.
 * Returns NOT_CONVERGED if eps_mbb > 0 was not reached within max_iters. */
EGT_API egt_status egt_solve(egt_game* game, const egt_solve_opts* opts, float* x_out, float* y_out,
                     egt_solve_report* rep, void* stream);

/* ---- batches: many games in one device-resident launch --------------------
 * A batch schedules games that the caller created and initialised
 * (egt_solver_init): each egt_batch_step is one cooperative launch whose CTAs
 * are split into groups; every group runs its members (games) in turn, each
 * for up to n_iters iterations of its own variant, stopping early at its own
 * eps_mbb target or max_iters (Alg. 1 / 3 loop test, residual every gap_every
 * iterations and at its last one).  A member's iterates are bit for bit those
 * egt_iterate gives it alone: its decisions come from fixed-order sums that do
 * not depend on the group size or on the other members.  The batch only reads
 * and advances its members' solver state; the games must outlive their
 * membership and must not be used by other calls while a step runs. */
typedef struct egt_batch egt_batch;

/* An empty batch on `device`. */
EGT_API egt_status egt_batch_create(int32_t device, egt_batch** out);
EGT_API egt_status egt_batch_destroy(egt_batch* batch);

/* Add an initialised game with opts->variant, eps_mbb, gap_every, max_iters
 * (max_iters counted from now; replay and log are not accepted).  *slot (host):
 * its index, stable until egt_batch_remove; freed slots are reused.  The
 * batch's launch arrays grow here (device and pinned host memory for the
 * members), so the steps allocate nothing.  OOM if that allocation fails. */
EGT_API egt_status egt_batch_add(egt_batch* batch, egt_game* game, const egt_solve_opts* opts,
                                 int32_t* slot);
EGT_API egt_status egt_batch_remove(egt_batch* batch, int32_t slot);

/* One launch advancing every active member by up to n_iters iterations.
 * group: CTAs per member, members dealt round-robin over the groups (0: the
 * batch's launch shape, egt_launch_shape below).  *n_active (host, may be
 * NULL): members still active afterwards.  A member stops being active when
 * it reaches its target (status OK), runs out of iterations (OK, or
 * NOT_CONVERGED if it had a target) or fails (its status). */
EGT_API egt_status egt_batch_step(egt_batch* batch, int32_t n_iters, int32_t group, int32_t* n_active,
                                  void* stream);

typedef struct {
  int32_t active;            /* 1 while the member still runs */
  int32_t status;            /* egt_status of the member */
  egt_solve_report rep;      /* since it was added: iterations, products, back-offs, residual
                                checks; the last residual, mu, tau; seconds = wall time of the
                                launches it took part in */
} egt_batch_member_info;

EGT_API egt_status egt_batch_member(const egt_batch* batch, int32_t slot, egt_batch_member_info* out);

/* Launch shape of the last egt_batch_step (of its last launch when it ran in waves): the widest
 * group's CTAs and the grid (host, either may be NULL). */
EGT_API egt_status egt_batch_launch_shape(const egt_batch* batch, int32_t* group, int32_t* grid);

/* How egt_batch_step (group = 0) splits the device over the active members.
 *   share:    0-4: CTAs per member in proportion to work^(share / 4), the work
 *             being the member's per-iteration cost (4: in proportion to it;
 *             0: equal shares; default 3, the best on a 64-game mix of 20- and
 *             52-card endgames); at least one CTA, at most the member's widest
 *             phase.  When the members outnumber the CTAs, one-CTA groups each
 *             run a least-loaded share of them (loads weighted the same way).
 *   pairs:    1 (default): a CTA runs two SBR / best-response / product items at
 *             a time, one per warp half, where shared memory allows and its group
 *             has two items per CTA; 0: one item at a time.
 *   grid_pct: percent of the co-resident CTAs launched, 1-100 (default 100).
 *   pack:     1: a makespan-balanced plan instead of share: members heavier than
 *             the balanced makespan get CTAs of their own in proportion to their
 *             work, the lighter ones share one-CTA groups that run them in turn
 *             (for batches with many small members); 0 (default): share.
 *   wave_mb:  > 0: the active members run in k = ceil(their device bytes
 *             (egt_dims.device_bytes) / wave_mb MB) consecutive waves of about
 *             equal bytes, one launch each, so that a wave's state can stay in
 *             L2 (default 128, about the B300's 126 MB L2); 0: all in one launch.
 *   wave_min: >= 1: at most (active members / wave_min) waves, at least one,
 *             so that every wave keeps about wave_min members: a wave of few
 *             members gives each of them many CTAs with few items apiece, the
 *             way one game alone runs, and loses more to that than L2 residency
 *             gains (default 16; 1: waves by bytes alone).
 * No choice changes any member's results (they come from exact products and
 * fixed-order sums); only the speed differs. */
typedef struct {
  int32_t share;
  int32_t pairs;
  int32_t grid_pct;
  int32_t pack;
  int32_t wave_mb;
  int32_t wave_min;
} egt_launch_shape;

/* Set / read the batch's launch shape (host structs).  Set returns
 * INVALID_ARG for a field outside the ranges above. */
EGT_API egt_status egt_batch_set_shape(egt_batch* batch, const egt_launch_shape* shape);
EGT_API egt_status egt_batch_get_shape(const egt_batch* batch, egt_launch_shape* shape);

#define EGT_TUNE_MAX 16

typedef struct {
  int32_t n;                            /* candidate shapes timed */
  int32_t best;                         /* index of the fastest (now the batch's shape), -1 if none */
  egt_launch_shape shape[EGT_TUNE_MAX];
  double us_per_iter[EGT_TUNE_MAX];     /* launch time (CUDA events) per member-iteration, best rep */
  int32_t iters[EGT_TUNE_MAX];          /* member-iterations of that rep */
} egt_tune_report;

/* Autotune the launch shape on the batch's own work: every candidate (share
 * 4 / 3 / 2 / 1 / 0 with pairs, share 4 / 3 / 2 without, share 3 on 75 % of
 * the CTAs, the packed plan, and share 3 in waves of 64 / 96 / 128 MB: 13
 * shapes) runs `reps` (>= 1) egt_batch_step
 * launches of n_iters iterations, each timed with CUDA events on `stream`, and
 * the shape with the least time per member-iteration becomes the batch's.  The
 * trials are real steps: members advance exactly as egt_batch_step advances
 * them and may finish while tuning.  A candidate that found no active member is
 * not timed (us_per_iter = 0, iters = 0); if none was timed the shape is
 * unchanged and best = -1.  rep (host) may be NULL. */
EGT_API egt_status egt_batch_tune(egt_batch* batch, int32_t n_iters, int32_t reps, egt_tune_report* rep,
                                  void* stream);

/* ---- serving: continuous batching of solve requests ------------------------
 * A server owns a batch on one device.  Requests (a game description and
 * solve options) wait in a FIFO queue; each egt_server_step admits queued
 * requests in order while their device memory (egt_dims.device_bytes) fits the
 * budget, runs one egt_batch_step over all running requests, and retires the
 * ones that stopped: their iterates are copied to host memory and their device
 * memory released.  Running requests keep x, y, mu on the device between
 * steps.  A request's result is bit for bit what egt_solve gives it alone. */
typedef struct egt_server egt_server;

typedef struct {
  int64_t mem_budget_bytes;   /* device memory for running requests; 0: 90 % of the free memory
                                 at creation (also the cap) */
  int32_t max_running;        /* 0: no cap besides memory */
  int32_t iters_per_step;     /* iterations per launch (0: 200) */
  int32_t group;              /* CTAs per request (0: automatic, see egt_batch_step) */
} egt_server_opts;

typedef struct {
  int32_t queued, running;
  int64_t completed, launches, used_bytes, budget_bytes;
  double clock;               /* seconds since the server was created */
} egt_server_stats;

typedef struct {
  int32_t state;              /* 0 queued, 1 running, 2 done */
  int32_t status;             /* egt_status once done (OK, NOT_CONVERGED, or the failure) */
  double t_submit, t_admit, t_done;   /* server clock (seconds); -1 if not yet */
  egt_solve_report rep;       /* once done: iterations, products, back-offs, residual, mu, tau */
  int32_t S[2], ld;           /* result layout: x [S[0]][ld], y [S[1]][ld] */
} egt_server_request_info;

/* opts (host) may be NULL (defaults). */
EGT_API egt_status egt_server_create(int32_t device, const egt_server_opts* opts, egt_server** out);
EGT_API egt_status egt_server_destroy(egt_server* server);

/* Seconds since the server was created (its clock for arrival and completion times). */
EGT_API double egt_server_clock(const egt_server* server);

/* Queue a request: the description is copied (the caller's arrays may be freed
 * after the call); opts: variant, alpha / mu0, eps_mbb, max_iters, gap_every
 * (replay and log are not accepted).  arrival: its arrival time on the server
 * clock (< 0: now), the origin of its latency.  *id (host): its handle.
 * OOM if the game alone exceeds the memory budget. */
EGT_API egt_status egt_server_submit(egt_server* server, const egt_game_desc* desc,
                                     const egt_solve_opts* opts, double arrival, int64_t* id);

/* Admit, run one launch over the running requests, retire the finished ones.
 * stats (host) may be NULL. */
EGT_API egt_status egt_server_step(egt_server* server, egt_server_stats* stats, void* stream);

/* State of a request; once done, its iterates are copied to x, y (host arrays
 * of S[0] x ld and S[1] x ld floats, either may be NULL) and, if release != 0,
 * the request is forgotten. */
EGT_API egt_status egt_server_result(egt_server* server, int64_t id, egt_server_request_info* info,
                                     float* x, float* y, int32_t release);

/* "queued", "running" or "done". */
EGT_API const char* egt_server_state_name(int32_t state);

/* ---- per-kernel device time accounting -------------------------------------- */

/* Kernel kinds of the accounting: FP32 product, FP64 product, smoothed best
 * response, FP64 best response, device-resident driver (egt_iterate). */
typedef enum {
  EGT_KERNEL_GRAD_F32 = 0,
  EGT_KERNEL_GRAD_F64 = 1,
  EGT_KERNEL_SBR = 2,
  EGT_KERNEL_BR_F64 = 3,
  EGT_KERNEL_ENGINE = 4,
  EGT_KERNEL_KINDS = 5
} egt_kernel_kind;

/* enable != 0: clear the totals and bracket every later kernel launch of this
 * game with CUDA events on its stream; enable == 0: stop timing.  Either call
 * restarts the launch counts (kept whether timing is on or off).  The events
 * add a little host work per launch. */
EGT_API egt_status egt_profile(egt_game* game, int32_t enable);

/* Device milliseconds per kernel kind timed since the last enable, and launches
 * per kind since the last egt_profile call (host arrays of EGT_KERNEL_KINDS
 * entries, either may be NULL).  Waits for the recorded launches to finish. */
EGT_API egt_status egt_profile_read(egt_game* game, double* ms, int64_t* launches);

/* Device time of the device-resident driver (egt_iterate / egt_solve, and the
 * game's batch steps) by phase, measured by CTA 0 while egt_profile timing is on
 * for the game (the clock reads cost about 2 % of the iteration rate, so they
 * are off otherwise) and summed since the last reset.  Phases: 0-5 the Step's
 * SBR / product / SBR / product / SBR / product phases (phase 0 is skipped when
 * the previous iteration computed this v_hat ahead; phase 5 then may carry the
 * next iteration's v_hat), 6 the phase after the Step (the other player's EGV
 * part, the residual's FP64 best responses, the next v_hat), 7 CTA 0's time
 * from the top of the iteration loop to its first phase (the fixed-order sums
 * of the per-item partials and the EGV / residual decisions when CTA 0 is the
 * group's deciding CTA, its last rank; the other CTAs start the next attempt
 * meanwhile), 8 from there to its first product phase.  phase_us: from
 * one mark to the next (for 0-6, barrier exits: the phase's slowest CTA and the
 * barrier included); work_us: for 0-6, from that exit to CTA 0's arrival at the
 * next barrier (its own items); phase_count: phases timed.  Host arrays of 9
 * entries, any may be NULL; reset != 0 clears the sums after reading. */
EGT_API egt_status egt_engine_trace(egt_game* game, int32_t reset, double* phase_us, double* work_us,
                                    int64_t* phase_count);

/* Message of the last failed call on this thread ("" if none). */
EGT_API const char* egt_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* EGT_H_ */
